// Vector kernels, the CG recurrence of Fig. 2 Alg. 1 and the C-ABI entry points.
//
// CG state lives in plan order on the device; scalars (r^H r, p^H q, step lengths,
// ||s||^2, history) are FP64. Reductions are deterministic: every kernel writes one
// partial per block and the last block to finish sums the partials in block order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sense_internal.cuh"
#include "sense_reduce.cuh"

namespace sense {

__device__ __forceinline__ bool stopped(const double* scal) { return scal[SC_STOP] != 0.0; }

// ---------------------------------------------------------------------------------------
// Layout kernels
// ---------------------------------------------------------------------------------------
__global__ void gather_image_kernel(const int32_t* __restrict__ perm, const float2* __restrict__ mu,
                                    float2* __restrict__ mp, int64_t Lp) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = perm[i];
    mp[i] = u >= 0 ? mu[u] : make_float2(0.f, 0.f);
  }
}

// out_user[perm[i]] = (sum_s src[s][i]) * (j if apply_j)
__global__ void scatter_kernel(const int32_t* __restrict__ perm, const float2* __restrict__ src,
                               int nsrc, int64_t Lp, const float* __restrict__ jv, int apply_j,
                               float2* __restrict__ mu) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = perm[i];
    if (u < 0) continue;
    float2 a = make_float2(0.f, 0.f);
    for (int s = 0; s < nsrc; ++s) {
      const float2 v = src[(int64_t)s * Lp + i];
      a.x += v.x;
      a.y += v.y;
    }
    if (apply_j) {
      a.x *= jv[i];
      a.y *= jv[i];
    }
    mu[u] = a;
  }
}

__global__ void load_data_kernel(const float2* __restrict__ su, int64_t K, int C, int64_t Kp,
                                 int Cp, float2* __restrict__ Y) {
  const int64_t n = Kp * Cp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / Cp;
    const int c = (int)(i % Cp);
    Y[i] = (k < K && c < C) ? su[k * C + c] : make_float2(0.f, 0.f);
  }
}

__global__ void reduce_xpart_kernel(const float2* __restrict__ Xpart, int nsplit, int64_t Lp,
                                    float2* __restrict__ q, const double* __restrict__ stop) {
  if (stop && *stop != 0.0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x) {
    float2 a = make_float2(0.f, 0.f);
    for (int s = 0; s < nsplit; ++s) {
      const float2 v = Xpart[(int64_t)s * Lp + i];
      a.x += v.x;
      a.y += v.y;
    }
    q[i] = a;
  }
}

// ---------------------------------------------------------------------------------------
// CG kernels (the CG loop of Alg. 1, Fig. 2)
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(VB) data_norm_kernel(const float2* __restrict__ Y, int64_t n,
                                                       double* part, unsigned* counter,
                                                       double* scal) {
  __shared__ double sh[1 * VB / 32];
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 y = Y[i];
    v[0] += (double)y.x * y.x + (double)y.y * y.y;
  }
  block_sum<1>(v, sh);
  double tot[1];
  if (finish_sums<1>(v, part, counter, tot)) scal[SC_SS] = tot[0];
}

// start: r = p = b, rho = 0; rr0 = b^H b; history row 0
__global__ void __launch_bounds__(VB) cg_init_kernel(const float2* __restrict__ b, float2* r,
                                                     float2* p, float2* x, int64_t Lp,
                                                     double* part, unsigned* counter,
                                                     double* scal, double* hist, double rel_tol,
                                                     int max_iter) {
  __shared__ double sh[1 * VB / 32];
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 bi = b[i];
    r[i] = bi;
    p[i] = bi;
    x[i] = make_float2(0.f, 0.f);
    v[0] += (double)bi.x * bi.x + (double)bi.y * bi.y;
  }
  block_sum<1>(v, sh);
  double tot[1];
  if (finish_sums<1>(v, part, counter, tot)) {
    scal[SC_RR] = tot[0];
    scal[SC_RR0] = tot[0];
    scal[SC_ITER] = 0.0;
    scal[SC_TOL2] = rel_tol > 0.0 ? rel_tol * rel_tol * tot[0] : 0.0;
    scal[SC_MAXIT] = (double)max_iter;
    // a zero residual (no data, or b = 0) is already the solution: stop as converged
    scal[SC_STOP] = (max_iter <= 0 || tot[0] == 0.0) ? 1.0 : (isfinite(tot[0]) ? 0.0 : 3.0);
    if (hist) {
      hist[0] = sqrt(tot[0]);
      hist[1] = 0.0;
      hist[2] = sqrt(scal[SC_SS]);
    }
  }
}

// start from rho_0 = x (plan order, already in place): with q = E^H E x, r = p = b - q;
// rr0 = r^H r, the tolerance relative to ||b||; history row 0 of the start
__global__ void __launch_bounds__(VB) cg_init_x0_kernel(const float2* __restrict__ b,
                                                        const float2* __restrict__ q,
                                                        const float2* __restrict__ x, float2* r,
                                                        float2* p, int64_t Lp, double* part,
                                                        unsigned* counter, double* scal,
                                                        double* hist, double rel_tol,
                                                        int max_iter) {
  __shared__ double sh[5 * VB / 32];
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 bi = b[i], qi = q[i], xi = x[i];
    const float2 ri = make_float2(bi.x - qi.x, bi.y - qi.y);
    r[i] = ri;
    p[i] = ri;
    v[0] += (double)ri.x * ri.x + (double)ri.y * ri.y;
    v[1] += (double)bi.x * bi.x + (double)bi.y * bi.y;
    v[2] += (double)xi.x * bi.x + (double)xi.y * bi.y;   // Re <x, b>
    v[3] += (double)xi.x * ri.x + (double)xi.y * ri.y;   // Re <x, r>
    v[4] += (double)xi.x * xi.x + (double)xi.y * xi.y;
  }
  block_sum<5>(v, sh);
  double tot[5];
  if (finish_sums<5>(v, part, counter, tot)) {
    scal[SC_RR] = tot[0];
    scal[SC_RR0] = tot[0];
    scal[SC_ITER] = 0.0;
    scal[SC_TOL2] = rel_tol > 0.0 ? rel_tol * rel_tol * tot[1] : 0.0;
    scal[SC_MAXIT] = (double)max_iter;
    const bool fin = isfinite(tot[0]) && isfinite(tot[4]);
    const bool done = max_iter <= 0 || tot[0] == 0.0 ||
                      (scal[SC_TOL2] > 0.0 && tot[0] <= scal[SC_TOL2]);
    scal[SC_STOP] = !fin ? 3.0 : (done ? 1.0 : 0.0);
    if (hist) {
      hist[0] = sqrt(tot[0]);
      hist[1] = sqrt(tot[4]);
      hist[2] = sqrt(fmax(0.0, scal[SC_SS] - tot[2] - tot[3]));
    }
  }
}

// alpha = r^H r, beta = p^H q and the step length alpha / beta
__global__ void __launch_bounds__(VB) cg_alpha_kernel(const float2* __restrict__ p,
                                                      const float2* __restrict__ q, int64_t Lp,
                                                      double* part, unsigned* counter,
                                                      double* scal) {
  if (stopped(scal)) return;
  __shared__ double sh[2 * VB / 32];
  double v[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = p[i], c = q[i];
    v[0] += (double)a.x * c.x + (double)a.y * c.y;   // Re conj(p) q
    v[1] += (double)a.x * c.y - (double)a.y * c.x;   // Im conj(p) q
  }
  block_sum<2>(v, sh);
  double tot[2];
  if (finish_sums<2>(v, part, counter, tot)) {
    scal[SC_PQ_RE] = tot[0];
    scal[SC_PQ_IM] = tot[1];
    const double den = tot[0] * tot[0] + tot[1] * tot[1];
    if (!(den > 0.0) || !isfinite(den)) {
      scal[SC_STOP] = isfinite(den) ? 2.0 : 3.0;
      return;
    }
    // alpha / beta with alpha = r^H r (real) and beta = p^H q (complex)
    const double rr = scal[SC_RR];
    scal[SC_A_RE] = rr * tot[0] / den;
    scal[SC_A_IM] = -rr * tot[1] / den;
  }
}

// rho += (alpha/beta) p, r -= (alpha/beta) q, the new r^H r and the history row of the new
// iterate
__global__ void __launch_bounds__(VB) cg_update_kernel(float2* x, float2* r,
                                                       const float2* __restrict__ p,
                                                       const float2* __restrict__ q,
                                                       const float2* __restrict__ b, int64_t Lp,
                                                       double* part, unsigned* counter,
                                                       double* scal, double* hist) {
  if (stopped(scal)) return;
  __shared__ double sh[4 * VB / 32];
  const float ar = (float)scal[SC_A_RE], ai = (float)scal[SC_A_IM];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 pi = p[i], qi = q[i], bi = b[i];
    float2 xi = x[i], ri = r[i];
    xi.x += ar * pi.x - ai * pi.y;
    xi.y += ar * pi.y + ai * pi.x;
    ri.x -= ar * qi.x - ai * qi.y;
    ri.y -= ar * qi.y + ai * qi.x;
    x[i] = xi;
    r[i] = ri;
    v[0] += (double)ri.x * ri.x + (double)ri.y * ri.y;
    v[1] += (double)xi.x * bi.x + (double)xi.y * bi.y;   // Re <x, b>
    v[2] += (double)xi.x * ri.x + (double)xi.y * ri.y;   // Re <x, r>
    v[3] += (double)xi.x * xi.x + (double)xi.y * xi.y;
  }
  block_sum<4>(v, sh);
  double tot[4];
  if (finish_sums<4>(v, part, counter, tot)) {
    const double rr_old = scal[SC_RR];
    scal[SC_RR_PREV] = rr_old;
    const double rr = tot[0];
    const int it = (int)scal[SC_ITER] + 1;
    scal[SC_ITER] = (double)it;
    if (hist) {
      hist[3 * it + 0] = sqrt(rr);
      hist[3 * it + 1] = sqrt(tot[3]);
      hist[3 * it + 2] = sqrt(fmax(0.0, scal[SC_SS] - tot[1] - tot[2]));
    }
    if (!isfinite(rr) || !isfinite(tot[3])) {
      scal[SC_STOP] = 3.0;
      return;
    }
    scal[SC_RR] = rr;
    scal[SC_B_RE] = rr / rr_old;   // alpha_new / beta with beta = alpha_old
    scal[SC_B_IM] = 0.0;
    if (scal[SC_TOL2] > 0.0 && rr <= scal[SC_TOL2]) scal[SC_STOP] = 1.0;
  }
}

// Residual replacement (van der Vorst and Ye): after the update of an iteration, the
// recursively updated residual is replaced by the true one, r = b - E^H E x, computed
// with the FP32 operator into q; the step-15 ratio and the history row are recomputed
// from it.
__global__ void __launch_bounds__(VB) cg_replace_kernel(const float2* __restrict__ x, float2* r,
                                                        const float2* __restrict__ b,
                                                        const float2* __restrict__ q,
                                                        int64_t Lp, double* part,
                                                        unsigned* counter, double* scal,
                                                        double* hist) {
  if (stopped(scal)) return;
  __shared__ double sh[3 * VB / 32];
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 bi = b[i], qi = q[i], xi = x[i];
    const float2 ri = make_float2(bi.x - qi.x, bi.y - qi.y);
    r[i] = ri;
    v[0] += (double)ri.x * ri.x + (double)ri.y * ri.y;
    v[1] += (double)xi.x * bi.x + (double)xi.y * bi.y;
    v[2] += (double)xi.x * ri.x + (double)xi.y * ri.y;
  }
  block_sum<3>(v, sh);
  double tot[3];
  if (finish_sums<3>(v, part, counter, tot)) {
    const int it = (int)scal[SC_ITER];
    const double rr = tot[0];
    if (hist) {
      hist[3 * it + 0] = sqrt(rr);
      hist[3 * it + 2] = sqrt(fmax(0.0, scal[SC_SS] - tot[1] - tot[2]));
    }
    if (!isfinite(rr)) {
      scal[SC_STOP] = 3.0;
      return;
    }
    scal[SC_RR] = rr;
    scal[SC_B_RE] = rr / scal[SC_RR_PREV];
    scal[SC_B_IM] = 0.0;
    if (scal[SC_TOL2] > 0.0 && rr <= scal[SC_TOL2]) scal[SC_STOP] = 1.0;
  }
}

// direction update p = r + (alpha_new / alpha_old) p
__global__ void cg_p_kernel(float2* p, const float2* __restrict__ r, int64_t Lp,
                            const double* scal) {
  if (stopped(scal)) return;
  const float br = (float)scal[SC_B_RE];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 pi = p[i], ri = r[i];
    p[i] = make_float2(ri.x + br * pi.x, ri.y + br * pi.y);
  }
}

// ---------------------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------------------
int grid_for(sense_plan_s* P, int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + VB - 1) / VB, 8 * P->num_sms));
}

int gather_image(sense_plan_s* P, const float2* mu, float2* mp, cudaStream_t st) {
  gather_image_kernel<<<grid_for(P, P->Lp), VB, 0, st>>>(P->dperm, mu, mp, P->Lp);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return SENSE_OK;
}

int scatter_xpart(sense_plan_s* P, float2* mu, bool apply_j, cudaStream_t st) {
  scatter_kernel<<<grid_for(P, P->Lp), VB, 0, st>>>(P->dperm, P->Xpart, P->nsplit_a, P->Lp, P->jv,
                                                    apply_j ? 1 : 0, mu);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return SENSE_OK;
}

int scatter_image(sense_plan_s* P, const float2* vp, float2* mu, bool apply_j, cudaStream_t st) {
  scatter_kernel<<<grid_for(P, P->Lp), VB, 0, st>>>(P->dperm, vp, 1, P->Lp, P->jv,
                                                    apply_j ? 1 : 0, mu);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return SENSE_OK;
}

int load_data(sense_plan_s* P, const float2* su, float2* Y, cudaStream_t st) {
  load_data_kernel<<<grid_for(P, P->Kp * P->Cp), VB, 0, st>>>(su, P->K, P->C, P->Kp, P->Cp, Y);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return SENSE_OK;
}

int reduce_xpart(sense_plan_s* P, float2* q, const double* stop, cudaStream_t st) {
  reduce_xpart_kernel<<<grid_for(P, P->Lp), VB, 0, st>>>(P->Xpart, P->nsplit_a, P->Lp, q, stop);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return SENSE_OK;
}

int check_prec(int prec) {
  if (prec == SENSE_PREC_FP32 || prec == SENSE_PREC_TC_FP16 || prec == SENSE_PREC_TC_SPLIT)
    return SENSE_OK;
  return set_error(SENSE_EINVAL, "unknown precision mode");
}

// q = E^H E p, all in plan order
int apply_normal_internal(sense_plan_s* P, int prec, const float2* p, float2* q,
                          const double* stop, cudaStream_t st) {
  int rc;
  NvtxRange nvtx("sense E^H E");
  if (prec != SENSE_PREC_FP32) {
    if ((rc = tc_encode(P, prec, p, P->Y, nullptr, true, stop, st)) != SENSE_OK) return rc;
    return tc_adjoint(P, prec, P->Y, q, true, stop, st);
  }
  if ((rc = fp32_encode_partials(P, p, stop, st)) != SENSE_OK) return rc;
  if ((rc = reduce_y(P, P->Y, nullptr, stop, st)) != SENSE_OK) return rc;
  if ((rc = fp32_adjoint_partials(P, P->Y, stop, st)) != SENSE_OK) return rc;
  return reduce_xpart(P, q, stop, st);
}

// q = E^H y for y in the internal data layout
int adjoint_internal(sense_plan_s* P, int prec, const float2* Y, float2* q, const double* stop,
                     cudaStream_t st) {
  int rc;
  if (prec != SENSE_PREC_FP32) return tc_adjoint(P, prec, Y, q, false, stop, st);
  if ((rc = fp32_adjoint_partials(P, Y, stop, st)) != SENSE_OK) return rc;
  return reduce_xpart(P, q, stop, st);
}

// one launch each of the step-length, update and direction kernels on the plan's CG vectors
int cg_step_alpha(sense_plan_s* P, cudaStream_t st) {
  cg_alpha_kernel<<<grid_for(P, P->Lp), VB, 0, st>>>(P->vp, P->vq, P->Lp, P->red, P->counter,
                                                     P->scal);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return SENSE_OK;
}

int cg_step_update(sense_plan_s* P, double* hist, cudaStream_t st) {
  cg_update_kernel<<<grid_for(P, P->Lp), VB, 0, st>>>(P->vx, P->vr, P->vp, P->vq, P->vb, P->Lp,
                                                      P->red, P->counter, P->scal, hist);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return SENSE_OK;
}

int cg_step_p(sense_plan_s* P, cudaStream_t st) {
  cg_p_kernel<<<grid_for(P, P->Lp), VB, 0, st>>>(P->vp, P->vr, P->Lp, P->scal);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return SENSE_OK;
}

// Y_int = E p (internal data layout)
int encode_internal(sense_plan_s* P, int prec, const float2* p, float2* Y, cudaStream_t st) {
  int rc;
  if (prec != SENSE_PREC_FP32) return tc_encode(P, prec, p, Y, nullptr, false, nullptr, st);
  if ((rc = fp32_encode_partials(P, p, nullptr, st)) != SENSE_OK) return rc;
  return reduce_y(P, Y, nullptr, nullptr, st);
}

// Argument staging: a host pointer is copied into a plan buffer (inputs) or written back
// after the work (outputs).

int stage_in(const void* user, void* buf, size_t bytes, cudaStream_t st, Staged* s) {
  s->user = user;
  s->host = !is_device_pointer(user);
  s->dev = s->host ? buf : const_cast<void*>(user);
  if (s->host)
    SENSE_CUDA_TRY(cudaMemcpyAsync(buf, user, bytes, cudaMemcpyHostToDevice, st));
  return SENSE_OK;
}

Staged stage_out(void* user, void* buf) {
  Staged s;
  s.user = user;
  s.host = !is_device_pointer(user);
  s.dev = s.host ? buf : user;
  return s;
}

int finish_out(const Staged& s, size_t bytes, cudaStream_t st) {
  if (!s.host) return SENSE_OK;
  SENSE_CUDA_TRY(cudaMemcpyAsync(const_cast<void*>(s.user), s.dev, bytes, cudaMemcpyDeviceToHost, st));
  SENSE_CUDA_TRY(cudaStreamSynchronize(st));
  return SENSE_OK;
}

int check_plan(sense_plan_s* P) {
  if (!P) return set_error(SENSE_EINVAL, "null plan");
  int dev = -1;
  SENSE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != P->device) return set_error(SENSE_EINVAL, "plan belongs to another device");
  return SENSE_OK;
}

}  // namespace sense

using namespace sense;

#define TRY(expr)                    \
  do {                               \
    int _rc = (expr);                \
    if (_rc != SENSE_OK) return _rc; \
  } while (0)

extern "C" int sense_encode(sense_plan P, int prec, const float* m, float* s, void* stream) {
  TRY(check_plan(P));
  if (!m || !s) return set_error(SENSE_EINVAL, "null m or s");
  TRY(check_prec(prec));
  cudaStream_t st = (cudaStream_t)stream;
  Staged in;
  TRY(stage_in(m, P->stage_m, (size_t)P->L * 8, st, &in));
  Staged out = stage_out(s, P->stage_s);
  TRY(gather_image(P, (const float2*)in.dev, P->vm, st));
  if (prec == SENSE_PREC_FP32) {
    TRY(fp32_encode_partials(P, P->vm, nullptr, st));
    TRY(reduce_y(P, nullptr, (float2*)out.dev, nullptr, st));
  } else {
    TRY(tc_encode(P, prec, P->vm, nullptr, (float2*)out.dev, false, nullptr, st));
  }
  TRY(finish_out(out, (size_t)P->K * P->C * 8, st));
  return out.host && prec != SENSE_PREC_FP32 ? tc_check_error(P) : SENSE_OK;
}

extern "C" int sense_adjoint(sense_plan P, int prec, const float* s, float* m, void* stream) {
  TRY(check_plan(P));
  if (!m || !s) return set_error(SENSE_EINVAL, "null m or s");
  TRY(check_prec(prec));
  cudaStream_t st = (cudaStream_t)stream;
  Staged in;
  TRY(stage_in(s, P->stage_s, (size_t)P->K * P->C * 8, st, &in));
  Staged out = stage_out(m, P->stage_m);
  TRY(load_data(P, (const float2*)in.dev, P->Y, st));
  if (prec == SENSE_PREC_FP32) {
    TRY(fp32_adjoint_partials(P, P->Y, nullptr, st));
    TRY(scatter_xpart(P, (float2*)out.dev, false, st));
  } else {
    TRY(tc_adjoint(P, prec, P->Y, P->vq, false, nullptr, st));
    TRY(scatter_image(P, P->vq, (float2*)out.dev, false, st));
  }
  TRY(finish_out(out, (size_t)P->L * 8, st));
  return out.host && prec != SENSE_PREC_FP32 ? tc_check_error(P) : SENSE_OK;
}

extern "C" int sense_normal_op(sense_plan P, int prec, const float* m, float* o, void* stream) {
  TRY(check_plan(P));
  if (!m || !o) return set_error(SENSE_EINVAL, "null m or out");
  TRY(check_prec(prec));
  cudaStream_t st = (cudaStream_t)stream;
  Staged in;
  TRY(stage_in(m, P->stage_m, (size_t)P->L * 8, st, &in));
  TRY(gather_image(P, (const float2*)in.dev, P->vm, st));
  Staged out = stage_out(o, P->stage_m);
  TRY(apply_normal_internal(P, prec, P->vm, P->vq, nullptr, st));
  TRY(scatter_image(P, P->vq, (float2*)out.dev, false, st));
  TRY(finish_out(out, (size_t)P->L * 8, st));
  return out.host && prec != SENSE_PREC_FP32 ? tc_check_error(P) : SENSE_OK;
}

extern "C" int sense_cg_solve_iterates(sense_plan P, const float* s, float* iterates,
                                       const sense_cg_opts* opts, double* history,
                                       sense_cg_info* info, void* stream) {
  TRY(check_plan(P));
  if (!s || !iterates || !opts) return set_error(SENSE_EINVAL, "null s, iterates or opts");
  if (opts->max_iter < 0 || !(opts->rel_tol >= 0.0) || opts->refine_every < 0)
    return set_error(SENSE_EINVAL, "max_iter, rel_tol and refine_every must be >= 0");
  TRY(check_prec(opts->prec));
  if (!is_device_pointer(iterates)) return set_error(SENSE_EINVAL, "iterates must be device memory");
  float2* X = (float2*)iterates;
  // the start rho_0 (use_x0) is read from row 0; the final iterate is row max_iter
  return cg_run(P, s, (float*)(X + (size_t)opts->max_iter * P->L), opts, history, info, 0,
                nullptr, X, (cudaStream_t)stream);
}

extern "C" int sense_cg_solve(sense_plan P, const float* s, float* x, const sense_cg_opts* opts,
                              double* history, sense_cg_info* info, void* stream) {
  TRY(check_plan(P));
  if (!s || !x || !opts) return set_error(SENSE_EINVAL, "null s, x or opts");
  if (opts->max_iter < 0 || !(opts->rel_tol >= 0.0) || opts->refine_every < 0)
    return set_error(SENSE_EINVAL, "max_iter, rel_tol and refine_every must be >= 0");
  TRY(check_prec(opts->prec));
  return cg_run(P, s, x, opts, history, info, 0, nullptr, nullptr, (cudaStream_t)stream);
}

namespace sense {

// Steps 1-5 for data s (device, user layout): coil data in the internal layout, ||s||^2,
// b = E^H s, x = 0 (or x = x0, device, user order, when x0 is given), r = p = b - E^H E x,
// r^H r and the stopping thresholds.
int cg_begin(sense_plan_s* P, const float2* s, const sense_cg_opts* opts, double* hist,
             cudaStream_t st, const float2* x0) {
  const int vb = grid_for(P, P->Lp);
  const int yb = grid_for(P, P->Kp * P->Cp);
  TRY(load_data(P, s, P->Ydata, st));
  data_norm_kernel<<<yb, VB, 0, st>>>(P->Ydata, P->Kp * P->Cp, P->red, P->counter, P->scal);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  // b = E^H sigma (FP32 operator, or the split tensor-core operator when the
  // iterations use it; FP32 whenever the residual is refined: b enters every replaced
  // residual)
  const int prec_b = (opts->prec == SENSE_PREC_TC_SPLIT && opts->refine_every == 0)
                         ? SENSE_PREC_TC_SPLIT
                         : SENSE_PREC_FP32;
  TRY(adjoint_internal(P, prec_b, P->Ydata, P->vb, nullptr, st));
  if (x0) {
    // r_0 = b - E^H E rho_0 with the operator b was made with
    TRY(gather_image(P, x0, P->vx, st));
    TRY(apply_normal_internal(P, prec_b, P->vx, P->vq, nullptr, st));
    cg_init_x0_kernel<<<vb, VB, 0, st>>>(P->vb, P->vq, P->vx, P->vr, P->vp, P->Lp, P->red,
                                         P->counter, P->scal, hist, opts->rel_tol,
                                         opts->max_iter);
  } else {
    cg_init_kernel<<<vb, VB, 0, st>>>(P->vb, P->vr, P->vp, P->vx, P->Lp, P->red, P->counter,
                                      P->scal, hist, opts->rel_tol, opts->max_iter);
  }
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return SENSE_OK;
}

// Synchronises st and reads the iteration count and status of the last solve.
int cg_read_info(sense_plan_s* P, sense_cg_info* info, int* iters, cudaStream_t st) {
  double sc[SC_COUNT];
  SENSE_CUDA_TRY(cudaMemcpyAsync(sc, P->scal, sizeof(sc), cudaMemcpyDeviceToHost, st));
  SENSE_CUDA_TRY(cudaStreamSynchronize(st));
  if (iters) *iters = (int)sc[SC_ITER];
  if (info) {
    info->iters = (int)sc[SC_ITER];
    info->status = sc[SC_STOP] == 2.0 ? SENSE_EBREAKDOWN
                   : sc[SC_STOP] == 3.0 ? SENSE_ENONFINITE
                                        : SENSE_OK;
    info->rr0 = sc[SC_RR0];
    info->rr_final = sc[SC_RR];
  }
  return SENSE_OK;
}

int cg_run(sense_plan_s* P, const float* s, float* x, const sense_cg_opts* opts,
           double* history, sense_cg_info* info, int ckpt_every, uint8_t* ckpt,
           float2* iterates, cudaStream_t st) {
  const int N = opts->max_iter;
  if (N + 1 > P->max_hist) {
    cudaFree(P->hist);
    P->hist = nullptr;
    if (cudaMalloc(&P->hist, (size_t)(N + 1) * 3 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      P->max_hist = 0;
      return set_error(SENSE_ENOMEM, "history buffer");
    }
    P->max_hist = N + 1;
  }
  Staged in;
  TRY(stage_in(s, P->stage_s, (size_t)P->K * P->C * 8, st, &in));
  // the start rho_0 (use_x0): from x, or from row 0 of the iterates; staged through the same
  // buffer as the result, which is written only after the start has been read
  const float2* x0 = nullptr;
  if (opts->use_x0) {
    if (iterates) {
      x0 = iterates;
    } else {
      Staged xin;
      TRY(stage_in(x, P->stage_m, (size_t)P->L * 8, st, &xin));
      x0 = (const float2*)xin.dev;
    }
  }
  Staged out = stage_out(x, P->stage_m);
  const int vb = grid_for(P, P->Lp);
  TRY(cg_begin(P, (const float2*)in.dev, opts, P->hist, st, x0));
  const double* stop = P->scal + SC_STOP;
  if (iterates && !x0) SENSE_CUDA_TRY(cudaMemsetAsync(iterates, 0, (size_t)P->L * 8, st));
  if (iterates && x0 && opts->apply_j) TRY(scatter_image(P, P->vx, iterates, true, st));
  for (int n = 0; n < N; ++n) {
    NvtxRange nvtx("sense CG iteration");
    if (ckpt_every > 0 && n % ckpt_every == 0) TRY(ckpt_save(P, ckpt, n / ckpt_every, st));
    // q = E^H E p
    TRY(apply_normal_internal(P, opts->prec, P->vp, P->vq, stop, st));
    TRY(cg_step_alpha(P, st));
    TRY(cg_step_update(P, P->hist, st));
    if (opts->prec != SENSE_PREC_FP32 && opts->refine_every > 0 &&
        (n + 1) % opts->refine_every == 0 && n + 1 < N) {
      // residual replacement with the FP32 operator
      TRY(apply_normal_internal(P, SENSE_PREC_FP32, P->vx, P->vm, stop, st));
      cg_replace_kernel<<<vb, VB, 0, st>>>(P->vx, P->vr, P->vb, P->vm, P->Lp, P->red,
                                           P->counter, P->scal, P->hist);
      SENSE_CUDA_TRY(cudaGetLastError());
      count_launch(P);
    }
    TRY(cg_step_p(P, st));
    // x_{n+1} in user order (after the stop it repeats the final iterate)
    if (iterates)
      TRY(scatter_image(P, P->vx, iterates + (size_t)(n + 1) * P->L, opts->apply_j != 0, st));
  }
  if (ckpt_every > 0) TRY(ckpt_final(P, ckpt, st));
  // rho <- rho o j
  TRY(scatter_image(P, P->vx, (float2*)out.dev, opts->apply_j != 0, st));
  if (history || info) {
    int iters = 0;
    TRY(cg_read_info(P, info, &iters, st));
    if (history)
      SENSE_CUDA_TRY(cudaMemcpy(history, P->hist, (size_t)(iters + 1) * 3 * sizeof(double),
                                cudaMemcpyDeviceToHost));
  }
  TRY(finish_out(out, (size_t)P->L * 8, st));
  const bool synced = history || info || out.host;
  return synced && opts->prec != SENSE_PREC_FP32 ? tc_check_error(P) : SENSE_OK;
}

}  // namespace sense
