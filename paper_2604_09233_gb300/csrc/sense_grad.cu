// Gradients with respect to the B0 map and the checkpointed, differentiable CG solve.
//
// B0 gradient. Row 0 of R is the B0 map omega (rad/s) and column 0 of K the sample time t,
// so d phi(kappa,l) / d omega(l) = t_kappa (Eq. 4). For a real loss with upstream gradient
// g = dL/dRe(y) + i dL/dIm(y):
//   y = E m     : dL/domega(l) = Im( conj(m(l))  (E^H (t o g))(l) ),   dL/dm = E^H g
//   x = E^H y   : dL/domega(l) = Im( conj(h(l))  (E^H (t o y))(l) ),   dL/dy = E h
// (h the upstream gradient of x). Both are the same primitive: a t-weighted adjoint followed
// by Im(conj(a) z) per voxel.
//
// CG backward. The forward follows Fig. 2 Alg. 1 with complex step length alpha = rho / gamma
// (rho = r^H r, gamma = p^H q), x' = x + alpha p, r' = r - alpha q, rho' = r'^H r',
// beta = rho' / rho, p' = r' + beta p, q = E^H E p. Reverse mode through one iteration, with
// gradients in the convention dL/dRe + i dL/dIm and xbar constant across iterations:
//   betabar  = Re <p, pbar'>
//   rbar'   += pbar' + 2 (rhobar' + betabar / rho) r'
//   alphabar = -<q, rbar'> + <p, xbar>
//   gammabar = -rho alphabar / conj(gamma)^2
//   rhobar   = -betabar rho' / rho^2 + Re(alphabar / conj(gamma))
//   qbar     = -conj(alpha) rbar' + gammabar p
//   pbar     = beta pbar' + conj(alpha) xbar + conj(gammabar) q + E^H E qbar
//   rbar     = rbar'
//   omegabar += Im(conj(p) E^H(t o E qbar)) + Im(conj(qbar) E^H(t o E p))
// and at the start (x_0 = 0, r_0 = p_0 = b, rho_0 = b^H b, b = E^H s):
//   bbar = rbar_0 + pbar_0 + 2 rhobar_0 b,  sbar = E bbar,  omegabar += Im(conj(bbar) E^H(t o s)).
// The forward stores r, p and its scalars every ckpt_every iterations; the backward replays
// each segment from its checkpoint (the kernels are deterministic, so the replay is
// bit-identical), keeping p_n, q_n, r_{n+1}, E p_n and the scalars of the segment, and then
// walks the segment backwards.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sense_internal.cuh"
#include "sense_reduce.cuh"

namespace sense {

namespace {

enum GradSlot { GS_BBAR = 0, GS_RHOBAR0, GS_RHOBAR1, GS_ABAR_RE, GS_ABAR_IM, GS_GBAR_RE,
                GS_GBAR_IM, GS_COUNT };

constexpr int32_t CKPT_MAGIC = 0x53434b31;  // "SCK1"

struct CkptHeader {
  int32_t magic, max_iter, every, prec, apply_j, pad0;
  int64_t Lp, nck;
  int64_t reserved[4];
};
static_assert(sizeof(CkptHeader) <= 256, "header fits its 256-byte slot");

int64_t round256(int64_t b) { return (b + 255) / 256 * 256; }
int64_t ckpt_slot_bytes(int64_t Lp) { return round256(2 * Lp * 8) + 256; }
int64_t ckpt_count(int max_iter, int every) { return max_iter / every + 1; }
int64_t ckpt_total_bytes(int64_t Lp, int max_iter, int every) {
  return 512 + ckpt_count(max_iter, every) * ckpt_slot_bytes(Lp);
}
// [0,256) header, [256,512) final scalars, then the slots: r [Lp], p [Lp], scalars
uint8_t* ckpt_slot(uint8_t* base, int64_t Lp, int64_t i) {
  return base + 512 + i * ckpt_slot_bytes(Lp);
}

__global__ void t_weight_kernel(const float2* __restrict__ Y, const float* __restrict__ tk,
                                int64_t n, int Cp, float2* __restrict__ Yt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float t = tk[i / Cp];
    const float2 v = Y[i];
    Yt[i] = make_float2(t * v.x, t * v.y);
  }
}

// gw = (acc ? gw : 0) + Im(conj(a) z)
__global__ void im_conj_kernel(const float2* __restrict__ a, const float2* __restrict__ z,
                               int64_t Lp, float* gw, int acc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 av = a[i], zv = z[i];
    const float v = av.x * zv.y - av.y * zv.x;
    gw[i] = acc ? gw[i] + v : v;
  }
}

__global__ void scatter_real_kernel(const int32_t* __restrict__ perm, const float* __restrict__ src,
                                    int64_t Lp, float* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = perm[i];
    if (u >= 0) dst[u] = src[i];
  }
}

// o = (mul_j ? j : 1) * v, plan order
__global__ void scale_j_kernel(const float2* __restrict__ v, const float* __restrict__ jv,
                               int64_t Lp, int mul_j, float2* __restrict__ o) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float w = mul_j ? jv[i] : 1.0f;
    o[i] = make_float2(w * v[i].x, w * v[i].y);
  }
}

// copies of up to three vectors and the scalar block (checkpoints, segment store)
__global__ void snapshot_kernel(const float2* __restrict__ a, const float2* __restrict__ b,
                                const float2* __restrict__ c, int64_t Lp, float2* __restrict__ da,
                                float2* __restrict__ db, float2* __restrict__ dc,
                                const double* __restrict__ scal, double* __restrict__ dscal) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (scal && tid < SC_COUNT) dscal[tid] = scal[tid];
  for (int64_t i = tid; i < Lp; i += (int64_t)gridDim.x * blockDim.x) {
    da[i] = a[i];
    db[i] = b[i];
    if (c) dc[i] = c[i];
  }
}

__global__ void zero_adjoints_kernel(float2* gr, float2* gp, float* gw, int64_t Lp,
                                     double* gsc) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid < GS_COUNT) gsc[tid] = 0.0;
  for (int64_t i = tid; i < Lp; i += (int64_t)gridDim.x * blockDim.x) {
    gr[i] = make_float2(0.f, 0.f);
    gp[i] = make_float2(0.f, 0.f);
    gw[i] = 0.f;
  }
}

// betabar = Re <p_n, pbar'>
__global__ void __launch_bounds__(VB) cgb_beta_kernel(const float2* __restrict__ p,
                                                      const float2* __restrict__ pbar, int64_t Lp,
                                                      double* part, unsigned* counter,
                                                      double* gsc) {
  __shared__ double sh[1 * VB / 32];
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = p[i], c = pbar[i];
    v[0] += (double)a.x * c.x + (double)a.y * c.y;
  }
  block_sum<1>(v, sh);
  double tot[1];
  if (finish_sums<1>(v, part, counter, tot)) gsc[GS_BBAR] = tot[0];
}

// rbar' += pbar' + 2 (rhobar' + betabar/rho) r'; then alphabar, gammabar, rhobar
__global__ void __launch_bounds__(VB) cgb_r_kernel(float2* rbar, const float2* __restrict__ pbar,
                                                   const float2* __restrict__ r1,
                                                   const float2* __restrict__ q,
                                                   const float2* __restrict__ p,
                                                   const float2* __restrict__ xbar, int64_t Lp,
                                                   const double* __restrict__ sc, double* part,
                                                   unsigned* counter, double* gsc, int rho_in,
                                                   int rho_out) {
  __shared__ double sh[4 * VB / 32];
  const double rho = sc[SC_RR_PREV], rho1 = sc[SC_RR];
  const double bbar = gsc[GS_BBAR];
  const float c = (float)(2.0 * (gsc[rho_in] + bbar / rho));
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 pb = pbar[i], rr = r1[i];
    float2 rb = rbar[i];
    rb.x += pb.x + c * rr.x;
    rb.y += pb.y + c * rr.y;
    rbar[i] = rb;
    const float2 qi = q[i], pi = p[i], xb = xbar[i];
    v[0] += (double)qi.x * rb.x + (double)qi.y * rb.y;   // <q, rbar>
    v[1] += (double)qi.x * rb.y - (double)qi.y * rb.x;
    v[2] += (double)pi.x * xb.x + (double)pi.y * xb.y;   // <p, xbar>
    v[3] += (double)pi.x * xb.y - (double)pi.y * xb.x;
  }
  block_sum<4>(v, sh);
  double tot[4];
  if (finish_sums<4>(v, part, counter, tot)) {
    const double ab_re = -tot[0] + tot[2], ab_im = -tot[1] + tot[3];
    // conj(gamma)
    const double gr = sc[SC_PQ_RE], gi = -sc[SC_PQ_IM];
    const double g2 = gr * gr + gi * gi;
    // alphabar / conj(gamma)
    const double u_re = (ab_re * gr + ab_im * gi) / g2, u_im = (ab_im * gr - ab_re * gi) / g2;
    // gammabar = -rho * (alphabar / conj(gamma)) / conj(gamma)
    gsc[GS_GBAR_RE] = -rho * (u_re * gr + u_im * gi) / g2;
    gsc[GS_GBAR_IM] = -rho * (u_im * gr - u_re * gi) / g2;
    gsc[GS_ABAR_RE] = ab_re;
    gsc[GS_ABAR_IM] = ab_im;
    gsc[rho_out] = -bbar * rho1 / (rho * rho) + u_re;
  }
}

// qbar = -conj(alpha) rbar + gammabar p;  pbar = beta pbar + conj(alpha) xbar + conj(gammabar) q
__global__ void cgb_q_kernel(const float2* __restrict__ rbar, float2* pbar,
                             const float2* __restrict__ xbar, const float2* __restrict__ p,
                             const float2* __restrict__ q, int64_t Lp,
                             const double* __restrict__ sc, const double* __restrict__ gsc,
                             float2* __restrict__ qbar) {
  const float ar = (float)sc[SC_A_RE], ai = -(float)sc[SC_A_IM];   // conj(alpha)
  const float beta = (float)sc[SC_B_RE];
  const float gr = (float)gsc[GS_GBAR_RE], gi = (float)gsc[GS_GBAR_IM];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 rb = rbar[i], pi = p[i], qi = q[i], xb = xbar[i];
    float2 pb = pbar[i];
    qbar[i] = make_float2(-(ar * rb.x - ai * rb.y) + (gr * pi.x - gi * pi.y),
                          -(ar * rb.y + ai * rb.x) + (gr * pi.y + gi * pi.x));
    // conj(gammabar) q
    const float cqx = gr * qi.x + gi * qi.y, cqy = gr * qi.y - gi * qi.x;
    pb.x = beta * pb.x + (ar * xb.x - ai * xb.y) + cqx;
    pb.y = beta * pb.y + (ar * xb.y + ai * xb.x) + cqy;
    pbar[i] = pb;
  }
}

// o += a
__global__ void add_kernel(float2* o, const float2* __restrict__ a, int64_t Lp) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x) {
    o[i].x += a[i].x;
    o[i].y += a[i].y;
  }
}

// bbar = rbar + pbar + 2 rhobar b
__global__ void cgb_b_kernel(const float2* __restrict__ rbar, const float2* __restrict__ pbar,
                             const float2* __restrict__ b, int64_t Lp,
                             const double* __restrict__ gsc, int rho_slot,
                             float2* __restrict__ bbar) {
  const float c = (float)(2.0 * gsc[rho_slot]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (int64_t)gridDim.x * blockDim.x)
    bbar[i] = make_float2(rbar[i].x + pbar[i].x + c * b[i].x, rbar[i].y + pbar[i].y + c * b[i].y);
}

template <typename T>
int dalloc_zero(T** p, size_t n) {
  if (cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_error(SENSE_ENOMEM, "gradient workspace");
  }
  return SENSE_OK;
}

#define GTRY(expr)                   \
  do {                               \
    int _rc = (expr);                \
    if (_rc != SENSE_OK) return _rc; \
  } while (0)

int grad_setup(sense_plan_s* P) {
  if (P->Yg) return SENSE_OK;
  const size_t ny = (size_t)P->Kp * P->Cp, nl = (size_t)P->Lp;
  int rc = SENSE_OK;
  if ((rc = dalloc_zero(&P->Yg, ny)) == SENSE_OK && (rc = dalloc_zero(&P->Yt, ny)) == SENSE_OK &&
      (rc = dalloc_zero(&P->vt, nl)) == SENSE_OK && (rc = dalloc_zero(&P->gw, nl)) == SENSE_OK &&
      (rc = dalloc_zero(&P->gx, nl)) == SENSE_OK && (rc = dalloc_zero(&P->gr, nl)) == SENSE_OK &&
      (rc = dalloc_zero(&P->gp, nl)) == SENSE_OK && (rc = dalloc_zero(&P->gq, nl)) == SENSE_OK &&
      (rc = dalloc_zero(&P->gsc, (size_t)GS_COUNT)) == SENSE_OK)
    return SENSE_OK;
  grad_free(P);
  return rc;
}

void seg_free(sense_plan_s* P) {
  cudaFree(P->seg_p); cudaFree(P->seg_q); cudaFree(P->seg_r); cudaFree(P->seg_Y);
  cudaFree(P->seg_sc);
  P->seg_p = P->seg_q = P->seg_r = P->seg_Y = nullptr;
  P->seg_sc = nullptr;
  P->seg_cap = 0;
}

int seg_setup(sense_plan_s* P, int cap) {
  if (P->seg_cap >= cap) return SENSE_OK;
  seg_free(P);
  const size_t nl = (size_t)P->Lp * cap, ny = (size_t)P->Kp * P->Cp * cap;
  int rc = SENSE_OK;
  if ((rc = dalloc_zero(&P->seg_p, nl)) == SENSE_OK && (rc = dalloc_zero(&P->seg_q, nl)) == SENSE_OK &&
      (rc = dalloc_zero(&P->seg_r, nl)) == SENSE_OK && (rc = dalloc_zero(&P->seg_Y, ny)) == SENSE_OK &&
      (rc = dalloc_zero(&P->seg_sc, (size_t)SC_COUNT * cap)) == SENSE_OK) {
    P->seg_cap = cap;
    return SENSE_OK;
  }
  seg_free(P);
  return rc;
}

// gw (+)= Im(conj(a) (E^H (t o Y))), all plan order / internal layout
int grad_b0_internal(sense_plan_s* P, int prec, const float2* a, const float2* Y, bool acc,
                     cudaStream_t st) {
  t_weight_kernel<<<grid_for(P, P->Kp * P->Cp), VB, 0, st>>>(Y, P->tk, P->Kp * P->Cp, P->Cp,
                                                             P->Yt);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  GTRY(adjoint_internal(P, prec, P->Yt, P->vt, nullptr, st));
  im_conj_kernel<<<grid_for(P, P->Lp), VB, 0, st>>>(a, P->vt, P->Lp, P->gw, acc ? 1 : 0);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return SENSE_OK;
}

int scatter_real(sense_plan_s* P, const float* src, float* dst, cudaStream_t st) {
  scatter_real_kernel<<<grid_for(P, P->Lp), VB, 0, st>>>(P->dperm, src, P->Lp, dst);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return SENSE_OK;
}

int snapshot(sense_plan_s* P, const float2* a, const float2* b, const float2* c, float2* da,
             float2* db, float2* dc, const double* scal, double* dscal, cudaStream_t st) {
  snapshot_kernel<<<grid_for(P, P->Lp), VB, 0, st>>>(a, b, c, P->Lp, da, db, dc, scal, dscal);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return SENSE_OK;
}

// Replays iterations n0 .. n1-1 from checkpoint ck (r, p, scalars) and keeps, per iteration
// i = n - n0, p_n, q_n, r_{n+1}, E p_n and the scalars after the update.
int replay_segment(sense_plan_s* P, int prec, uint8_t* ck, int n0, int n1, cudaStream_t st) {
  const int64_t Lp = P->Lp;
  const float2* cr = (const float2*)ck;
  const float2* cp = cr + Lp;
  const double* csc = (const double*)(ck + round256(2 * Lp * 8));
  SENSE_CUDA_TRY(cudaMemcpyAsync(P->vr, cr, Lp * 8, cudaMemcpyDeviceToDevice, st));
  SENSE_CUDA_TRY(cudaMemcpyAsync(P->vp, cp, Lp * 8, cudaMemcpyDeviceToDevice, st));
  SENSE_CUDA_TRY(cudaMemcpyAsync(P->scal, csc, SC_COUNT * 8, cudaMemcpyDeviceToDevice, st));
  // x does not enter the replayed quantities; it only has to stay finite
  SENSE_CUDA_TRY(cudaMemsetAsync(P->vx, 0, Lp * 8, st));
  const double* stop = P->scal + SC_STOP;
  for (int n = n0; n < n1; ++n) {
    const int i = n - n0;
    GTRY(apply_normal_internal(P, prec, P->vp, P->vq, stop, st));
    GTRY(cg_step_alpha(P, st));
    GTRY(cg_step_update(P, nullptr, st));
    GTRY(snapshot(P, P->vp, P->vq, P->vr, P->seg_p + i * Lp, P->seg_q + i * Lp,
                  P->seg_r + i * Lp, P->scal, P->seg_sc + (int64_t)i * SC_COUNT, st));
    SENSE_CUDA_TRY(cudaMemcpyAsync(P->seg_Y + (int64_t)i * P->Kp * P->Cp, P->Y,
                                   (size_t)P->Kp * P->Cp * 8, cudaMemcpyDeviceToDevice, st));
    GTRY(cg_step_p(P, st));
  }
  return SENSE_OK;
}

}  // namespace

void grad_free(sense_plan_s* P) {
  cudaFree(P->Yg); cudaFree(P->Yt); cudaFree(P->vt); cudaFree(P->gw);
  cudaFree(P->gx); cudaFree(P->gr); cudaFree(P->gp); cudaFree(P->gq); cudaFree(P->gsc);
  P->Yg = P->Yt = P->vt = nullptr;
  P->gw = nullptr;
  P->gx = P->gr = P->gp = P->gq = nullptr;
  P->gsc = nullptr;
  seg_free(P);
}

int ckpt_save(sense_plan_s* P, uint8_t* ckpt, int64_t slot, cudaStream_t st) {
  uint8_t* s = ckpt_slot(ckpt, P->Lp, slot);
  float2* r = (float2*)s;
  return snapshot(P, P->vr, P->vp, nullptr, r, r + P->Lp, nullptr, P->scal,
                  (double*)(s + round256(2 * P->Lp * 8)), st);
}

int ckpt_final(sense_plan_s* P, uint8_t* ckpt, cudaStream_t st) {
  SENSE_CUDA_TRY(cudaMemcpyAsync(ckpt + 256, P->scal, SC_COUNT * 8, cudaMemcpyDeviceToDevice, st));
  return SENSE_OK;
}

}  // namespace sense

using namespace sense;

extern "C" int sense_grad_b0(sense_plan P, int prec, const float* a, const float* y, float* z,
                             float* grad_omega, void* stream) {
  GTRY(check_plan(P));
  if (!a || !y || !grad_omega) return set_error(SENSE_EINVAL, "null a, y or grad_omega");
  GTRY(check_prec(prec));
  GTRY(grad_setup(P));
  cudaStream_t st = (cudaStream_t)stream;
  Staged in;
  GTRY(stage_in(y, P->stage_s, (size_t)P->K * P->C * 8, st, &in));
  GTRY(load_data(P, (const float2*)in.dev, P->Yg, st));
  bool synced = in.host;
  if (z) {
    Staged zo = stage_out(z, P->stage_m);
    GTRY(adjoint_internal(P, prec, P->Yg, P->vq, nullptr, st));
    GTRY(scatter_image(P, P->vq, (float2*)zo.dev, false, st));
    GTRY(finish_out(zo, (size_t)P->L * 8, st));
    synced = synced || zo.host;
  }
  Staged ain;
  GTRY(stage_in(a, P->stage_m, (size_t)P->L * 8, st, &ain));
  GTRY(gather_image(P, (const float2*)ain.dev, P->gx, st));
  GTRY(grad_b0_internal(P, prec, P->gx, P->Yg, false, st));
  Staged go = stage_out(grad_omega, P->stage_m);
  GTRY(scatter_real(P, P->gw, (float*)go.dev, st));
  GTRY(finish_out(go, (size_t)P->L * 4, st));
  synced = synced || go.host;
  return synced && prec != SENSE_PREC_FP32 ? tc_check_error(P) : SENSE_OK;
}

extern "C" int64_t sense_cg_ckpt_bytes(sense_plan P, int32_t max_iter, int32_t ckpt_every) {
  if (!P) return set_error(SENSE_EINVAL, "null plan");
  if (max_iter < 0 || ckpt_every < 1)
    return set_error(SENSE_EINVAL, "max_iter must be >= 0 and ckpt_every >= 1");
  return ckpt_total_bytes(P->Lp, max_iter, ckpt_every);
}

extern "C" int sense_cg_solve_ckpt(sense_plan P, const float* s, float* x,
                                   const sense_cg_opts* opts, int32_t ckpt_every, void* ckpt,
                                   int64_t ckpt_bytes, sense_cg_info* info, void* stream) {
  GTRY(check_plan(P));
  if (!s || !x || !opts || !ckpt) return set_error(SENSE_EINVAL, "null s, x, opts or ckpt");
  if (opts->max_iter < 0 || !(opts->rel_tol >= 0.0) || ckpt_every < 1)
    return set_error(SENSE_EINVAL, "max_iter, rel_tol must be >= 0 and ckpt_every >= 1");
  if (opts->refine_every != 0)
    return set_error(SENSE_EINVAL, "checkpointed solves do not support residual replacement");
  if (opts->use_x0)
    return set_error(SENSE_EINVAL, "checkpointed solves start from rho = 0 (use_x0 must be 0)");
  GTRY(check_prec(opts->prec));
  if (!is_device_pointer(ckpt) || ((uintptr_t)ckpt & 15))
    return set_error(SENSE_EINVAL, "ckpt must be 16-byte aligned device memory");
  if (ckpt_bytes < ckpt_total_bytes(P->Lp, opts->max_iter, ckpt_every))
    return set_error(SENSE_EINVAL, "ckpt_bytes below sense_cg_ckpt_bytes()");
  cudaStream_t st = (cudaStream_t)stream;
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  h.magic = CKPT_MAGIC;
  h.max_iter = opts->max_iter;
  h.every = ckpt_every;
  h.prec = opts->prec;
  h.apply_j = opts->apply_j != 0;
  h.Lp = P->Lp;
  h.nck = ckpt_count(opts->max_iter, ckpt_every);
  // pageable source: the copy has read h when the call returns
  SENSE_CUDA_TRY(cudaMemcpyAsync(ckpt, &h, sizeof(h), cudaMemcpyHostToDevice, st));
  return cg_run(P, s, x, opts, nullptr, info, ckpt_every, (uint8_t*)ckpt, nullptr, st);
}

extern "C" int sense_cg_backward(sense_plan P, const float* s, const void* ckpt,
                                 int64_t ckpt_bytes, const float* xbar, float* sbar,
                                 float* omega_bar, void* stream) {
  GTRY(check_plan(P));
  if (!s || !ckpt || !xbar || (!sbar && !omega_bar))
    return set_error(SENSE_EINVAL, "null s, ckpt or xbar, or no output");
  if (!is_device_pointer(ckpt) || ((uintptr_t)ckpt & 15))
    return set_error(SENSE_EINVAL, "ckpt must be 16-byte aligned device memory");
  if (ckpt_bytes < 512) return set_error(SENSE_EINVAL, "ckpt_bytes too small");
  cudaStream_t st = (cudaStream_t)stream;
  uint8_t head[512];
  SENSE_CUDA_TRY(cudaMemcpyAsync(head, ckpt, sizeof(head), cudaMemcpyDeviceToHost, st));
  SENSE_CUDA_TRY(cudaStreamSynchronize(st));
  CkptHeader h;
  std::memcpy(&h, head, sizeof(h));
  double fsc[SC_COUNT];
  std::memcpy(fsc, head + 256, sizeof(fsc));
  if (h.magic != CKPT_MAGIC || h.Lp != P->Lp || h.every < 1 ||
      ckpt_bytes < ckpt_total_bytes(P->Lp, h.max_iter, h.every))
    return set_error(SENSE_EINVAL, "ckpt was not written by sense_cg_solve_ckpt on this plan");
  const int iters = (int)fsc[SC_ITER];
  if (iters < 0 || iters > h.max_iter)
    return set_error(SENSE_EINVAL, "ckpt holds no finished solve");
  const int prec = h.prec, every = h.every;
  GTRY(grad_setup(P));
  GTRY(seg_setup(P, every));
  const int64_t Lp = P->Lp, ny = P->Kp * P->Cp;
  const int vb = grid_for(P, Lp);
  uint8_t* ck = (uint8_t*)const_cast<void*>(ckpt);

  // inputs: s into the data layout, xbar into plan order (times j when x was scaled by j)
  Staged sin_, xin;
  GTRY(stage_in(s, P->stage_s, (size_t)P->K * P->C * 8, st, &sin_));
  GTRY(load_data(P, (const float2*)sin_.dev, P->Ydata, st));
  GTRY(stage_in(xbar, P->stage_m, (size_t)P->L * 8, st, &xin));
  GTRY(gather_image(P, (const float2*)xin.dev, P->gx, st));
  scale_j_kernel<<<vb, VB, 0, st>>>(P->gx, P->jv, Lp, h.apply_j, P->gx);
  SENSE_CUDA_TRY(cudaGetLastError());
  zero_adjoints_kernel<<<vb, VB, 0, st>>>(P->gr, P->gp, P->gw, Lp, P->gsc);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P, 2);

  int rho_in = GS_RHOBAR0, rho_out = GS_RHOBAR1;
  for (int c = iters > 0 ? (iters - 1) / every : -1; c >= 0; --c) {
    const int n0 = c * every, n1 = std::min(n0 + every, iters);
    GTRY(replay_segment(P, prec, ckpt_slot(ck, Lp, c), n0, n1, st));
    for (int n = n1 - 1; n >= n0; --n) {
      const int64_t i = n - n0;
      const float2* pn = P->seg_p + i * Lp;
      const float2* qn = P->seg_q + i * Lp;
      const float2* r1 = P->seg_r + i * Lp;
      const double* sc = P->seg_sc + i * SC_COUNT;
      cgb_beta_kernel<<<vb, VB, 0, st>>>(pn, P->gp, Lp, P->red, P->counter, P->gsc);
      SENSE_CUDA_TRY(cudaGetLastError());
      cgb_r_kernel<<<vb, VB, 0, st>>>(P->gr, P->gp, r1, qn, pn, P->gx, Lp, sc, P->red,
                                      P->counter, P->gsc, rho_in, rho_out);
      SENSE_CUDA_TRY(cudaGetLastError());
      cgb_q_kernel<<<vb, VB, 0, st>>>(P->gr, P->gp, P->gx, pn, qn, Lp, sc, P->gsc, P->gq);
      SENSE_CUDA_TRY(cudaGetLastError());
      count_launch(P, 3);
      // pbar += E^H E qbar; omegabar += Im(conj(p) E^H(t o E qbar)) + Im(conj(qbar) E^H(t o E p))
      GTRY(encode_internal(P, prec, P->gq, P->Yg, st));
      GTRY(adjoint_internal(P, prec, P->Yg, P->vt, nullptr, st));
      add_kernel<<<vb, VB, 0, st>>>(P->gp, P->vt, Lp);
      SENSE_CUDA_TRY(cudaGetLastError());
      count_launch(P);
      GTRY(grad_b0_internal(P, prec, pn, P->Yg, true, st));
      GTRY(grad_b0_internal(P, prec, P->gq, P->seg_Y + i * ny, true, st));
      std::swap(rho_in, rho_out);
    }
  }

  // b = E^H s with the operator the solve used for it
  const int prec_b = prec == SENSE_PREC_TC_SPLIT ? SENSE_PREC_TC_SPLIT : SENSE_PREC_FP32;
  Staged so = stage_out(sbar, P->stage_s);
  Staged wo = stage_out(omega_bar, P->stage_m);
  if (iters > 0) {
    const float2* b = (const float2*)ckpt_slot(ck, Lp, 0);   // r_0 = b
    cgb_b_kernel<<<vb, VB, 0, st>>>(P->gr, P->gp, b, Lp, P->gsc, rho_in, P->gq);
    SENSE_CUDA_TRY(cudaGetLastError());
    count_launch(P);
    if (sbar) {
      if (prec_b == SENSE_PREC_FP32) {
        GTRY(fp32_encode_partials(P, P->gq, nullptr, st));
        GTRY(reduce_y(P, nullptr, (float2*)so.dev, nullptr, st));
      } else {
        GTRY(tc_encode(P, prec_b, P->gq, nullptr, (float2*)so.dev, false, nullptr, st));
      }
    }
    if (omega_bar) GTRY(grad_b0_internal(P, prec_b, P->gq, P->Ydata, true, st));
  } else if (sbar) {
    SENSE_CUDA_TRY(cudaMemsetAsync(so.dev, 0, (size_t)P->K * P->C * 8, st));
  }
  if (sbar) GTRY(finish_out(so, (size_t)P->K * P->C * 8, st));
  if (omega_bar) {
    GTRY(scatter_real(P, P->gw, (float*)wo.dev, st));
    GTRY(finish_out(wo, (size_t)P->L * 4, st));
  }
  const bool synced = (sbar && so.host) || (omega_bar && wo.host);
  return synced && prec != SENSE_PREC_FP32 ? tc_check_error(P) : SENSE_OK;
}
