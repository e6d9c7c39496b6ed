// Diagnostics: per-launch event timing, launch counting, and a sincos-throughput probe
// used as the special-function-unit roof of the on-the-fly encoding kernels.
#include <algorithm>
#include <utility>

#include "sense_internal.cuh"

namespace sense {

int prof_begin(sense_plan_s* P, int kc, cudaStream_t st) {
  if (!P->prof_on) return SENSE_OK;
  if (P->prof_used == P->prof_events.size()) {
    cudaEvent_t a, b;
    SENSE_CUDA_TRY(cudaEventCreate(&a));
    SENSE_CUDA_TRY(cudaEventCreate(&b));
    P->prof_events.push_back({kc, {a, b}});
  }
  auto& e = P->prof_events[P->prof_used];
  e.first = kc;
  SENSE_CUDA_TRY(cudaEventRecord(e.second.first, st));
  return SENSE_OK;
}

int prof_end(sense_plan_s* P, cudaStream_t st) {
  if (!P->prof_on) return SENSE_OK;
  SENSE_CUDA_TRY(cudaEventRecord(P->prof_events[P->prof_used].second.second, st));
  ++P->prof_used;
  return SENSE_OK;
}

void prof_free(sense_plan_s* P) {
  for (auto& e : P->prof_events) {
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
  P->prof_events.clear();
  P->prof_used = 0;
}

// Each thread runs 8 independent sincos chains; one chain step = one __sincosf plus one
// FMA to carry the dependency.
__global__ void sincos_probe_kernel(int iters, float* sink) {
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = 0.001f * (threadIdx.x + 37 * j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float s, c;
      __sincosf(x[j], &s, &c);
      x[j] = fmaf(s, 0.75f, c);
    }
  }
  float a = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) a += x[j];
  if (a == 12345.678f) sink[threadIdx.x] = a;  // practically never; keeps the chains live
}

}  // namespace sense

using namespace sense;

extern "C" int sense_plan_sync(sense_plan P, void* stream) {
  if (!P) return set_error(SENSE_EINVAL, "null plan");
  SENSE_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  return tc_check_error(P);
}

extern "C" int sense_plan_get_tuning(sense_plan P, sense_tuning* out) {
  if (!P || !out) return set_error(SENSE_EINVAL, "null plan or output");
  *out = sense_tuning{};
  out->seg_len = P->tc_seg_len;
  out->grid = P->tc_grid_req == P->num_sms ? 0 : P->tc_grid_req;
  out->wait_limit_us = P->tc_wait_us;
  out->test_hold_stage = P->tc_test_hold;
  out->inner_chunk = P->tc_inner_chunk;
  return SENSE_OK;
}

extern "C" int sense_plan_set_tuning(sense_plan P, const sense_tuning* t) {
  if (!P || !t) return set_error(SENSE_EINVAL, "null plan or tuning");
  if (t->wait_limit_us < 0 || t->wait_limit_us > 60000000 || t->test_hold_stage < 0 ||
      t->inner_chunk < 0)
    return set_error(SENSE_EINVAL,
                     "wait_limit_us must be 0..6e7, test_hold_stage and inner_chunk >= 0");
  const int rc = tc_set_tuning(P, t->seg_len, t->grid, t->inner_chunk);
  if (rc != SENSE_OK) return rc;
  P->tc_wait_us = t->wait_limit_us;
  P->tc_wait_cycles = (long long)t->wait_limit_us * (P->clock_khz / 1000);
  P->tc_test_hold = t->test_hold_stage;
  return SENSE_OK;
}

extern "C" int sense_plan_profile(sense_plan P, int enable) {
  if (!P) return set_error(SENSE_EINVAL, "null plan");
  P->prof_on = enable != 0;
  P->prof_used = 0;
  P->n_launch = 0;
  return SENSE_OK;
}

extern "C" int sense_plan_stats(sense_plan P, sense_stats* out) {
  if (!P || !out) return set_error(SENSE_EINVAL, "null plan or output");
  *out = sense_stats{};
  out->launches = P->n_launch;
  for (size_t i = 0; i < P->prof_used; ++i) {
    auto& e = P->prof_events[i];
    SENSE_CUDA_TRY(cudaEventSynchronize(e.second.second));
    float ms = 0.f;
    SENSE_CUDA_TRY(cudaEventElapsedTime(&ms, e.second.first, e.second.second));
    out->timed[e.first] += 1;
    out->ms[e.first] += ms;
  }
  return SENSE_OK;
}

extern "C" int sense_diag_sincos_rate(double ms_budget, double* per_s) {
  if (!per_s || !(ms_budget > 0.0)) return set_error(SENSE_EINVAL, "bad arguments");
  int dev = 0, sms = 0;
  SENSE_CUDA_TRY(cudaGetDevice(&dev));
  SENSE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  float* sink = nullptr;
  SENSE_CUDA_TRY(cudaMalloc(&sink, 1024 * sizeof(float)));
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int blocks = sms * 8, threads = 256;
  int iters = 256;
  float ms = 0.f;
  // warm up and scale the iteration count to the budget
  for (int round = 0; round < 6; ++round) {
    cudaEventRecord(a);
    sincos_probe_kernel<<<blocks, threads>>>(iters, sink);
    cudaEventRecord(b);
    SENSE_CUDA_TRY(cudaEventSynchronize(b));
    cudaEventElapsedTime(&ms, a, b);
    if (ms > 0.5 * ms_budget) break;
    iters = (int)std::min<double>(1 << 22, iters * std::max(2.0, 0.9 * ms_budget / std::max(ms, 0.01f)));
  }
  cudaEventRecord(a);
  sincos_probe_kernel<<<blocks, threads>>>(iters, sink);
  cudaEventRecord(b);
  SENSE_CUDA_TRY(cudaEventSynchronize(b));
  cudaEventElapsedTime(&ms, a, b);
  SENSE_CUDA_TRY(cudaGetLastError());
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  *per_s = (double)blocks * threads * 8.0 * iters / (ms * 1e-3);
  return SENSE_OK;
}
