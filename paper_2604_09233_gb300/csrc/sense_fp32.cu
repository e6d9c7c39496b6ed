// FP32 CUDA-core ("explicit") E and E^H.
//
// Both kernels evaluate the phase of each (sample, voxel) pair once and reuse the
// exponential for every coil, as in Eq. 4 / Eq. 5 written as P (S o m 1^T) and
// (S* o P^H Sigma) 1. One thread owns one row of the pair tile (a sample for E, a voxel
// for E^H) and all coils of it; the other dimension streams through shared memory in
// sub-blocks of 64, with its per-column data read by broadcast. The contraction over the
// streamed dimension is split across CTAs (deterministic partial buffers, reduced in a
// fixed order afterwards).
#include <algorithm>

#include "sense_internal.cuh"

namespace sense {

constexpr int SUB = 64;  // streamed sub-block

template <int RP>
__device__ __forceinline__ float phase_turns(float base, const float* __restrict__ own,
                                             const float* __restrict__ other) {
  float th = 0.0f;
#pragma unroll
  for (int q = 0; q < RP; q += 4) {
    const float4 o = *reinterpret_cast<const float4*>(other + q);
    th = fmaf(own[q + 0], o.x, th);
    th = fmaf(own[q + 1], o.y, th);
    th = fmaf(own[q + 2], o.z, th);
    th = fmaf(own[q + 3], o.w, th);
  }
  th += base;
  return th - rintf(th);
}

// E: Ypart[split][k][c] = sum_{l in split} e^{+i 2pi th(k,l)} S(l,c) m(l)
template <int CP, int RP>
__global__ void __launch_bounds__(TILE) encode_f32_kernel(
    const float* __restrict__ dK, const float* __restrict__ dR, const float* __restrict__ Aanc,
    const float* __restrict__ Banc, const float2* __restrict__ S, const float2* __restrict__ m,
    float2* __restrict__ Ypart, int64_t Lp, int64_t Kp, int nvb, int vb_per_split,
    const double* __restrict__ stop) {
  if (stop && *stop != 0.0) return;
  __shared__ __align__(16) float sR[SUB * RP];
  __shared__ float sA[SUB];
  __shared__ float2 sQ[SUB * CP];
  const int sb = blockIdx.x, split = blockIdx.y, t = threadIdx.x;
  const int64_t k = (int64_t)sb * TILE + t;
  float own[RP];
#pragma unroll
  for (int q = 0; q < RP; q += 4) {
    const float4 v = *reinterpret_cast<const float4*>(dK + k * RP + q);
    own[q] = v.x; own[q + 1] = v.y; own[q + 2] = v.z; own[q + 3] = v.w;
  }
  float2 acc[CP];
#pragma unroll
  for (int c = 0; c < CP; ++c) acc[c] = make_float2(0.f, 0.f);
  const int vb0 = split * vb_per_split;
  const int vb1 = min(nvb, vb0 + vb_per_split);
  for (int vb = vb0; vb < vb1; ++vb) {
    const float bk = Banc[(int64_t)vb * Kp + k];
    for (int h = 0; h < TILE / SUB; ++h) {
      const int64_t l0 = (int64_t)vb * TILE + h * SUB;
      __syncthreads();
      for (int i = t; i < SUB * RP; i += TILE) sR[i] = dR[l0 * RP + i];
      if (t < SUB) sA[t] = Aanc[(int64_t)sb * Lp + l0 + t];
      for (int i = t; i < SUB * CP; i += TILE) {
        const int v = i / CP;
        const float2 s = S[(l0 + v) * CP + (i % CP)];
        const float2 mv = m[l0 + v];
        sQ[i] = make_float2(s.x * mv.x - s.y * mv.y, s.x * mv.y + s.y * mv.x);
      }
      __syncthreads();
#pragma unroll 2
      for (int v = 0; v < SUB; ++v) {
        const float th = phase_turns<RP>(sA[v] + bk, own, sR + v * RP);
        float sn, cs;
        __sincosf(6.283185307179586f * th, &sn, &cs);
#pragma unroll
        for (int c = 0; c < CP; ++c) {
          const float2 q = sQ[v * CP + c];
          acc[c].x = fmaf(cs, q.x, fmaf(-sn, q.y, acc[c].x));
          acc[c].y = fmaf(cs, q.y, fmaf(sn, q.x, acc[c].y));
        }
      }
    }
  }
  float2* out = Ypart + ((int64_t)split * Kp + k) * CP;
#pragma unroll
  for (int c = 0; c < CP; ++c) out[c] = acc[c];
}

// E^H (before the coil sum): Xpart[split][l] = sum_c conj(S(l,c)) sum_{k in split}
//   e^{-i 2pi th(k,l)} Y(k,c)
template <int CP, int RP>
__global__ void __launch_bounds__(TILE) adjoint_f32_kernel(
    const float* __restrict__ dK, const float* __restrict__ dR, const float* __restrict__ Aanc,
    const float* __restrict__ Banc, const float2* __restrict__ S, const float2* __restrict__ Y,
    float2* __restrict__ Xpart, int64_t Lp, int64_t Kp, int nsb, int sb_per_split,
    const double* __restrict__ stop) {
  if (stop && *stop != 0.0) return;
  __shared__ __align__(16) float sK[SUB * RP];
  __shared__ float sB[SUB];
  __shared__ float2 sY[SUB * CP];
  const int vb = blockIdx.x, split = blockIdx.y, t = threadIdx.x;
  const int64_t l = (int64_t)vb * TILE + t;
  float own[RP];
#pragma unroll
  for (int q = 0; q < RP; q += 4) {
    const float4 v = *reinterpret_cast<const float4*>(dR + l * RP + q);
    own[q] = v.x; own[q + 1] = v.y; own[q + 2] = v.z; own[q + 3] = v.w;
  }
  float2 acc[CP];
#pragma unroll
  for (int c = 0; c < CP; ++c) acc[c] = make_float2(0.f, 0.f);
  const int sb0 = split * sb_per_split;
  const int sb1 = min(nsb, sb0 + sb_per_split);
  for (int sb = sb0; sb < sb1; ++sb) {
    const float al = Aanc[(int64_t)sb * Lp + l];
    for (int h = 0; h < TILE / SUB; ++h) {
      const int64_t k0 = (int64_t)sb * TILE + h * SUB;
      __syncthreads();
      for (int i = t; i < SUB * RP; i += TILE) sK[i] = dK[k0 * RP + i];
      if (t < SUB) sB[t] = Banc[(int64_t)vb * Kp + k0 + t];
      for (int i = t; i < SUB * CP; i += TILE) sY[i] = Y[k0 * CP + i];
      __syncthreads();
#pragma unroll 2
      for (int kk = 0; kk < SUB; ++kk) {
        const float th = phase_turns<RP>(al + sB[kk], own, sK + kk * RP);
        float sn, cs;
        __sincosf(6.283185307179586f * th, &sn, &cs);
#pragma unroll
        for (int c = 0; c < CP; ++c) {
          const float2 y = sY[kk * CP + c];
          acc[c].x = fmaf(cs, y.x, fmaf(sn, y.y, acc[c].x));
          acc[c].y = fmaf(cs, y.y, fmaf(-sn, y.x, acc[c].y));
        }
      }
    }
  }
  float2 v = make_float2(0.f, 0.f);
#pragma unroll
  for (int c = 0; c < CP; ++c) {
    const float2 s = S[l * CP + c];
    v.x = fmaf(s.x, acc[c].x, fmaf(s.y, acc[c].y, v.x));
    v.y = fmaf(s.x, acc[c].y, fmaf(-s.y, acc[c].x, v.y));
  }
  Xpart[(int64_t)split * Lp + l] = v;
}

// Y_int[k][c] = sum_split Ypart (0 for padded samples); optionally also s_user[k][c<C].
__global__ void reduce_y_kernel(const float2* __restrict__ Ypart, int nsplit, int64_t K,
                                int64_t Kp, int C, int Cp, float2* __restrict__ Y_int,
                                float2* __restrict__ s_user, const double* __restrict__ stop) {
  if (stop && *stop != 0.0) return;
  const int64_t n = Kp * Cp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / Cp;
    const int c = (int)(i % Cp);
    float2 a = make_float2(0.f, 0.f);
    if (k < K && c < C)
      for (int s = 0; s < nsplit; ++s) {
        const float2 v = Ypart[(int64_t)s * n + i];
        a.x += v.x;
        a.y += v.y;
      }
    if (Y_int) Y_int[i] = a;
    if (s_user && k < K && c < C) s_user[k * C + c] = a;
  }
}

template <int CP, int RP>
static void launch_encode(sense_plan_s* P, const float2* m, const double* stop, cudaStream_t st) {
  encode_f32_kernel<CP, RP><<<dim3(P->nsb, P->nsplit_e), TILE, 0, st>>>(
      P->dK, P->dR, P->Aanc, P->Banc, P->S, m, P->Ypart, P->Lp, P->Kp, P->nvb, P->vb_per_split,
      stop);
}

template <int CP, int RP>
static void launch_adjoint(sense_plan_s* P, const float2* Y, const double* stop,
                           cudaStream_t st) {
  adjoint_f32_kernel<CP, RP><<<dim3(P->nvb, P->nsplit_a), TILE, 0, st>>>(
      P->dK, P->dR, P->Aanc, P->Banc, P->S, Y, P->Xpart, P->Lp, P->Kp, P->nsb, P->sb_per_split,
      stop);
}

#define SENSE_DISPATCH_RP(FN, CPV, ...)                       \
  switch (P->RP) {                                            \
    case 4: FN<CPV, 4>(__VA_ARGS__); break;                   \
    case 8: FN<CPV, 8>(__VA_ARGS__); break;                   \
    case 12: FN<CPV, 12>(__VA_ARGS__); break;                 \
    case 16: FN<CPV, 16>(__VA_ARGS__); break;                 \
    default: FN<CPV, 20>(__VA_ARGS__); break;                 \
  }
#define SENSE_DISPATCH(FN, ...)                                 \
  switch (P->Cp) {                                              \
    case 8: SENSE_DISPATCH_RP(FN, 8, __VA_ARGS__); break;       \
    case 16: SENSE_DISPATCH_RP(FN, 16, __VA_ARGS__); break;     \
    case 32: SENSE_DISPATCH_RP(FN, 32, __VA_ARGS__); break;     \
    default: SENSE_DISPATCH_RP(FN, 64, __VA_ARGS__); break;     \
  }

int fp32_encode_partials(sense_plan_s* P, const float2* m_plan, const double* stop,
                         cudaStream_t st) {
  int rc = prof_begin(P, KC_F32_ENC, st);
  if (rc != SENSE_OK) return rc;
  SENSE_DISPATCH(launch_encode, P, m_plan, stop, st);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return prof_end(P, st);
}

int fp32_adjoint_partials(sense_plan_s* P, const float2* Y_int, const double* stop,
                          cudaStream_t st) {
  int rc = prof_begin(P, KC_F32_ADJ, st);
  if (rc != SENSE_OK) return rc;
  SENSE_DISPATCH(launch_adjoint, P, Y_int, stop, st);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return prof_end(P, st);
}

int reduce_y(sense_plan_s* P, float2* Y_int, float2* s_user, const double* stop,
             cudaStream_t st) {
  const int64_t n = P->Kp * P->Cp;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8 * P->num_sms);
  reduce_y_kernel<<<blocks, 256, 0, st>>>(P->Ypart, P->nsplit_e, P->K, P->Kp, P->C, P->Cp,
                                          Y_int, s_user, stop);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return SENSE_OK;
}

}  // namespace sense
