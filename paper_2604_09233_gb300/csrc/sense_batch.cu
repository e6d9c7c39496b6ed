// Batched reconstruction: many independent problems of uneven size (matrix, coils, samples,
// field-expansion order) solved together.
//
// Every E and E^H of a batch iteration is ONE persistent launch of the tensor-core pass
// kernel over all instances: the work is a queue of items (instance, row block, chunk of
// streamed blocks) that CTAs claim with an atomic counter, so large and small instances
// share the GPU and an instance whose CG has stopped drops out of the queue (its items are
// skipped) without leaving CTAs idle. Each item writes its own partial slot (slot = chunk),
// summed in a fixed order afterwards, so results are deterministic. All instances use one
// kernel instantiation: their plans are built with the batch-wide padded coil count and
// delta-row count (zero padding).
//
// One CG iteration of the whole batch (images, the two batched passes, the per-instance
// reductions and CG vector kernels) is captured once in a CUDA graph and replayed; the
// per-instance stop flags turn finished instances' kernels into no-ops.
//
// The chunk length (streamed blocks per work item) and the accumulator segment length are
// chosen by sense_batch_autotune, which times the batched E^H E for each candidate.
#include <algorithm>
#include <vector>

#include "sense_tc.cuh"

struct sense_batch_s {
  int device = 0, num_sms = 0;
  std::vector<sense_plan_s*> plans;
  int Cp = 8, RT = 4;
  int chunk = 16, seg_len = 4;
  // per mode (ENC, ADJ): descriptors with / without the CG stop flag, and the work items
  sense::tc::InstDesc* desc[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  int4* items[2] = {nullptr, nullptr};
  int n_items[2] = {0, 0};
  unsigned* qnext = nullptr;       // [2] claim counters
  int* err = nullptr;              // time-out word of the batched passes
  std::vector<float2*> ypart, xpart;   // per instance [nchunk][Kp][Cp], [nchunk][Lp][xpart coils]
  std::vector<int*> nslot_e, nslot_a;  // per instance, per row block: nchunk
  cudaGraphExec_t gexec = nullptr;
  int graph_prec = -1;
  std::vector<int64_t> geom_versions;  // of each plan when the descriptors were built
  // side streams for the instances' small kernels, and the events that fork them from and
  // join them back into the caller's stream (a set per fork site of one CG iteration)
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> events;   // [FORK_SITES][1 + side.size()]
};

namespace sense {
namespace {

constexpr int CHUNK_CANDIDATES[] = {8, 16, 32, 64};
constexpr int MAX_SIDE_STREAMS = 16;
constexpr int FORK_SITES = 3;  // per CG iteration: B images of p; Y and its image; reduction + CG

// Run fn(b, stream) for every instance b, spread round-robin over the batch's side streams,
// which wait for everything issued on st so far; st then waits for all of them. The instances'
// small kernels (a few blocks each) so run concurrently instead of one after another, and in a
// captured CUDA graph they form parallel branches. `site` selects the events of this fork.
template <class F>
int for_instances(sense_batch_s* B, int site, cudaStream_t st, F&& fn) {
  const int n = (int)B->plans.size();
  const int S = (int)B->side.size();
  if (S == 0) {
    for (int b = 0; b < n; ++b) {
      const int rc = fn(b, st);
      if (rc != SENSE_OK) return rc;
    }
    return SENSE_OK;
  }
  cudaEvent_t* ev = &B->events[(size_t)site * (1 + S)];
  SENSE_CUDA_TRY(cudaEventRecord(ev[0], st));
  for (int k = 0; k < S; ++k) SENSE_CUDA_TRY(cudaStreamWaitEvent(B->side[k], ev[0], 0));
  int rc = SENSE_OK;
  for (int b = 0; b < n && rc == SENSE_OK; ++b) rc = fn(b, B->side[b % S]);
  // join even after a failure, so that no side stream is left outside a capture
  for (int k = 0; k < S; ++k) {
    SENSE_CUDA_TRY(cudaEventRecord(ev[1 + k], B->side[k]));
    SENSE_CUDA_TRY(cudaStreamWaitEvent(st, ev[1 + k], 0));
  }
  return rc;
}

int create_side_streams(sense_batch_s* B) {
  const int S = std::min<int>((int)B->plans.size(), MAX_SIDE_STREAMS);
  if (S < 2) return SENSE_OK;
  for (int k = 0; k < S; ++k) {
    cudaStream_t s;
    SENSE_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    B->side.push_back(s);
  }
  for (int e = 0; e < FORK_SITES * (1 + S); ++e) {
    cudaEvent_t ev;
    SENSE_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    B->events.push_back(ev);
  }
  return SENSE_OK;
}
constexpr int SEG_CANDIDATES[] = {2, 4};

int dmalloc(void** p, size_t bytes, const char* what) {
  if (cudaMalloc(p, std::max<size_t>(bytes, 1)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_error(SENSE_ENOMEM, what);
  }
  return SENSE_OK;
}

void free_layout(sense_batch_s* B) {
  for (int m = 0; m < 2; ++m) {
    cudaFree(B->desc[m][0]);
    cudaFree(B->desc[m][1]);
    cudaFree(B->items[m]);
    B->desc[m][0] = B->desc[m][1] = nullptr;
    B->items[m] = nullptr;
    B->n_items[m] = 0;
  }
  for (auto* p : B->ypart) cudaFree(p);
  for (auto* p : B->xpart) cudaFree(p);
  for (auto* p : B->nslot_e) cudaFree(p);
  for (auto* p : B->nslot_a) cudaFree(p);
  B->ypart.clear();
  B->xpart.clear();
  B->nslot_e.clear();
  B->nslot_a.clear();
  if (B->gexec) cudaGraphExecDestroy(B->gexec);
  B->gexec = nullptr;
  B->graph_prec = -1;
}

// Work items, partial buffers and descriptors for the current chunk length.
int build_layout(sense_batch_s* B) {
  free_layout(B);
  const int n = (int)B->plans.size();
  B->geom_versions.clear();
  for (auto* P : B->plans) {
    // a rebuilt geometry (sense_plan_set_b0 on a member plan) must keep the batch layout
    if (P->Cp != B->Cp || P->RT != B->RT)
      return set_error(SENSE_EUNSUPPORTED, "a member plan left the batch-wide layout");
    B->geom_versions.push_back(P->geom_version);
  }
  const int CH = B->chunk;
  std::vector<int4> it[2];
  std::vector<tc::InstDesc> d[2][2];
  int rc;
  for (int b = 0; b < n; ++b) {
    sense_plan_s* P = B->plans[b];
    const int nch_e = (P->nvb + CH - 1) / CH, nch_a = (P->nsb + CH - 1) / CH;
    float2 *yp = nullptr, *xp = nullptr;
    int *ne = nullptr, *na = nullptr;
    if ((rc = dmalloc((void**)&yp, (size_t)nch_e * P->Kp * P->Cp * 8, "batch partials")) ||
        (B->ypart.push_back(yp), 0) ||
        (rc = dmalloc((void**)&xp, (size_t)nch_a * P->Lp * tc_xpart_coils(P) * 8,
                      "batch partials")) ||
        (B->xpart.push_back(xp), 0) ||
        (rc = dmalloc((void**)&ne, (size_t)P->nsb * 4, "batch slots")) ||
        (B->nslot_e.push_back(ne), 0) ||
        (rc = dmalloc((void**)&na, (size_t)P->nvb * 4, "batch slots")) ||
        (B->nslot_a.push_back(na), 0))
      return rc;
    std::vector<int> ve((size_t)P->nsb, nch_e), va((size_t)P->nvb, nch_a);
    SENSE_CUDA_TRY(cudaMemcpy(ne, ve.data(), ve.size() * 4, cudaMemcpyHostToDevice));
    SENSE_CUDA_TRY(cudaMemcpy(na, va.data(), va.size() * 4, cudaMemcpyHostToDevice));
    for (int m = 0; m < 2; ++m) {
      const bool enc = m == tc::ENC;
      tc::InstDesc e = {};
      e.rowT = enc ? P->dKt : P->dRt;
      e.colT = enc ? P->dRt : P->dKt;
      e.rowAnc = enc ? P->Banc : P->Aanc;
      e.colAnc = enc ? P->Aanc : P->Banc;
      e.Bimg = enc ? P->Qimg : P->Yimg;
      e.bscale = enc ? P->qscale : P->yscale;
      e.S = P->S;
      e.out = enc ? yp : xp;
      e.rows_total = enc ? P->Kp : P->Lp;
      e.cols_total = enc ? P->Lp : P->Kp;
      e.n_outer = enc ? P->nsb : P->nvb;
      e.n_inner = enc ? P->nvb : P->nsb;
      e.chunk = CH;
      e.rowPh = enc ? P->phK_row : P->phR_row;
      e.colPh = enc ? P->phR_col : P->phK_col;
      e.rowAncR = enc ? P->BancR : P->AancR;
      e.colAncR = enc ? P->AancR : P->BancR;
      e.ph_unscale = P->ph_unscale;
      e.stop = nullptr;
      d[m][0].push_back(e);
      e.stop = P->scal + SC_STOP;
      d[m][1].push_back(e);
      for (int o = 0; o < e.n_outer; ++o)
        for (int c0 = 0; c0 < e.n_inner; c0 += CH)
          it[m].push_back(make_int4(b, o, c0, std::min(c0 + CH, e.n_inner)));
    }
  }
  for (int m = 0; m < 2; ++m) {
    for (int s = 0; s < 2; ++s) {
      if ((rc = dmalloc((void**)&B->desc[m][s], d[m][s].size() * sizeof(tc::InstDesc),
                        "batch descriptors")))
        return rc;
      SENSE_CUDA_TRY(cudaMemcpy(B->desc[m][s], d[m][s].data(),
                                d[m][s].size() * sizeof(tc::InstDesc), cudaMemcpyHostToDevice));
    }
    if ((rc = dmalloc((void**)&B->items[m], it[m].size() * sizeof(int4), "batch items")))
      return rc;
    SENSE_CUDA_TRY(cudaMemcpy(B->items[m], it[m].data(), it[m].size() * sizeof(int4),
                              cudaMemcpyHostToDevice));
    B->n_items[m] = (int)it[m].size();
  }
  return SENSE_OK;
}

int batch_pass(sense_batch_s* B, int mode, int npart, bool with_stop, cudaStream_t st) {
  SENSE_CUDA_TRY(cudaMemsetAsync(B->qnext + mode, 0, 4, st));
  tc::Params prm = {};
  prm.inst = B->desc[mode][with_stop ? 1 : 0];
  prm.items = B->items[mode];
  prm.n_items = B->n_items[mode];
  prm.next = B->qnext + mode;
  prm.first_cta = nullptr;
  prm.W = 0;
  prm.err = B->err;
  prm.stop = nullptr;
  prm.seg_len = B->seg_len;
  return tc_launch(B->plans[0], mode, npart, B->Cp, B->RT, prm, B->num_sms, st);
}

// q_b = E_b^H E_b p_b for every instance b (plan-order vectors of each plan); with_stop:
// instances whose CG has stopped are skipped.
int batch_normal(sense_batch_s* B, int prec, const std::vector<const float2*>& p,
                 const std::vector<float2*>& q, bool with_stop, cudaStream_t st,
                 bool reduce_x = true) {
  const int np = prec == SENSE_PREC_TC_SPLIT ? 2 : 1;
  int rc;
  if ((rc = for_instances(B, 0, st, [&](int b, cudaStream_t s) {
         sense_plan_s* P = B->plans[b];
         return tc_make_image(P, np, nullptr, p[b], P->Lp, P->colmax, P->qscale, P->Qimg, false,
                              s);
       })))
    return rc;
  if ((rc = batch_pass(B, tc::ENC, np, with_stop, st))) return rc;
  if ((rc = for_instances(B, 1, st, [&](int b, cudaStream_t s) {
         sense_plan_s* P = B->plans[b];
         const double* stop = with_stop ? P->scal + SC_STOP : nullptr;
         int r = tc_reduce_y(P, B->ypart[b], B->nslot_e[b], P->Y, nullptr, P->colmax + P->Cp,
                             stop, s);
         if (r == SENSE_OK)
           r = tc_make_image(P, np, P->Y, nullptr, P->Kp, P->colmax + P->Cp, P->yscale, P->Yimg,
                             true, s);
         return r;
       })))
    return rc;
  if ((rc = batch_pass(B, tc::ADJ, np, with_stop, st))) return rc;
  if (!reduce_x) return SENSE_OK;
  return for_instances(B, 2, st, [&](int b, cudaStream_t s) {
    sense_plan_s* P = B->plans[b];
    const double* stop = with_stop ? P->scal + SC_STOP : nullptr;
    return tc_reduce_x(P, B->xpart[b], B->nslot_a[b], q[b], stop, s);
  });
}

// one CG iteration (E^H E p, step length, updates, direction) of every instance
int batch_cg_iteration(sense_batch_s* B, int prec, cudaStream_t st) {
  std::vector<const float2*> p;
  std::vector<float2*> q;
  for (auto* P : B->plans) {
    p.push_back(P->vp);
    q.push_back(P->vq);
  }
  int rc;
  if ((rc = batch_normal(B, prec, p, q, true, st, false))) return rc;
  // per instance: the E^H reduction into q, then the CG step length, updates and direction
  return for_instances(B, 2, st, [&](int b, cudaStream_t s) {
    sense_plan_s* P = B->plans[b];
    int r = tc_reduce_x(P, B->xpart[b], B->nslot_a[b], q[b], P->scal + SC_STOP, s);
    if (r == SENSE_OK) r = cg_step_alpha(P, s);
    if (r == SENSE_OK) r = cg_step_update(P, nullptr, s);
    if (r == SENSE_OK) r = cg_step_p(P, s);
    return r;
  });
}

int check_err(sense_batch_s* B) {
  int e = 0;
  SENSE_CUDA_TRY(cudaMemcpy(&e, B->err, 4, cudaMemcpyDeviceToHost));
  if (e != 0) {
    cudaMemset(B->err, 0, 4);
    return set_error(SENSE_ETIMEOUT, "batched tensor-core pass timed out waiting (site " +
                                         std::to_string(e) + ")");
  }
  return SENSE_OK;
}

int check_batch(sense_batch_s* B) {
  if (!B) return set_error(SENSE_EINVAL, "null batch");
  int dev = -1;
  SENSE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != B->device) return set_error(SENSE_EINVAL, "batch belongs to another device");
  // the descriptors hold the plans' geometry pointers: rebuild them after a member plan's
  // geometry was rebuilt (its B0 map replaced)
  for (size_t b = 0; b < B->plans.size(); ++b)
    if (b >= B->geom_versions.size() || B->plans[b]->geom_version != B->geom_versions[b]) {
      SENSE_CUDA_TRY(cudaDeviceSynchronize());
      return build_layout(B);
    }
  return SENSE_OK;
}

void batch_free(sense_batch_s* B) {
  if (!B) return;
  free_layout(B);
  for (auto s : B->side) cudaStreamDestroy(s);
  for (auto e : B->events) cudaEventDestroy(e);
  cudaFree(B->qnext);
  cudaFree(B->err);
  for (auto* P : B->plans) sense_plan_destroy(P);
  delete B;
}

}  // namespace
}  // namespace sense

using namespace sense;

#define BTRY(expr)                   \
  do {                               \
    int _rc = (expr);                \
    if (_rc != SENSE_OK) return _rc; \
  } while (0)

extern "C" int sense_batch_create(const sense_problem* probs, int32_t n, sense_batch* out) {
  if (!probs || !out || n < 1) return set_error(SENSE_EINVAL, "null problems/output or n < 1");
  *out = nullptr;
  // batch-wide padded coils and delta rows: build each plan once to learn its own, then
  // rebuild the smaller ones with the batch-wide values
  sense_batch_s* B = new sense_batch_s();
  int rc = SENSE_OK;
  std::vector<sense_plan_s*> first((size_t)n, nullptr);
  for (int b = 0; b < n && rc == SENSE_OK; ++b) rc = plan_create(&probs[b], 0, 0, &first[b]);
  if (rc == SENSE_OK) {
    for (auto* P : first) {
      B->Cp = std::max(B->Cp, P->Cp);
      B->RT = std::max(B->RT, P->RT);
    }
    for (int b = 0; b < n && rc == SENSE_OK; ++b) {
      if (first[b]->Cp == B->Cp && first[b]->RT == B->RT) {
        B->plans.push_back(first[b]);
        first[b] = nullptr;
      } else {
        sense_plan_s* P = nullptr;
        rc = plan_create(&probs[b], B->Cp, B->RT, &P);
        if (rc == SENSE_OK) B->plans.push_back(P);
      }
    }
  }
  for (auto* P : first) sense_plan_destroy(P);
  if (rc == SENSE_OK) {
    B->device = B->plans[0]->device;
    B->num_sms = B->plans[0]->num_sms;
    for (auto* P : B->plans)
      if (P->Cp != B->Cp || P->RT != B->RT) rc = set_error(SENSE_EUNSUPPORTED, "uniform layout");
  }
  if (rc == SENSE_OK) rc = dmalloc((void**)&B->qnext, 8, "batch counters");
  if (rc == SENSE_OK) rc = dmalloc((void**)&B->err, 4, "batch error word");
  if (rc == SENSE_OK && cudaMemset(B->err, 0, 4) != cudaSuccess)
    rc = cuda_error(cudaGetLastError(), "cudaMemset");
  if (rc == SENSE_OK) rc = build_layout(B);
  if (rc == SENSE_OK) rc = create_side_streams(B);
  if (rc != SENSE_OK) {
    batch_free(B);
    return rc;
  }
  *out = B;
  return SENSE_OK;
}

extern "C" int sense_batch_destroy(sense_batch B) {
  if (!B) return SENSE_OK;
  cudaDeviceSynchronize();
  batch_free(B);
  return SENSE_OK;
}

extern "C" int sense_batch_plan(sense_batch B, int32_t i, sense_plan* out) {
  if (!B || !out || i < 0 || i >= (int)B->plans.size())
    return set_error(SENSE_EINVAL, "null batch/output or index out of range");
  *out = B->plans[i];
  return SENSE_OK;
}

extern "C" int sense_batch_info(sense_batch B, int32_t out[4]) {
  if (!B || !out) return set_error(SENSE_EINVAL, "null batch or output");
  out[0] = (int32_t)B->plans.size();
  out[1] = B->Cp;
  out[2] = B->RT;
  out[3] = B->chunk;
  return SENSE_OK;
}

extern "C" int sense_batch_normal_op(sense_batch B, int32_t prec, const float* const* m,
                                     float* const* o, void* stream) {
  BTRY(check_batch(B));
  if (!m || !o) return set_error(SENSE_EINVAL, "null vector arrays");
  if (prec != SENSE_PREC_TC_FP16 && prec != SENSE_PREC_TC_SPLIT)
    return set_error(SENSE_EINVAL, "batched operators run on the tensor cores (TC_FP16, TC_SPLIT)");
  const int n = (int)B->plans.size();
  for (int b = 0; b < n; ++b)
    if (!m[b] || !o[b] || !is_device_pointer(m[b]) || !is_device_pointer(o[b]))
      return set_error(SENSE_EINVAL, "batched vectors must be device pointers");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<const float2*> p;
  std::vector<float2*> q;
  for (int b = 0; b < n; ++b) {
    sense_plan_s* P = B->plans[b];
    BTRY(gather_image(P, (const float2*)m[b], P->vm, st));
    p.push_back(P->vm);
    q.push_back(P->vq);
  }
  BTRY(batch_normal(B, prec, p, q, false, st));
  for (int b = 0; b < n; ++b) BTRY(scatter_image(B->plans[b], B->plans[b]->vq, (float2*)o[b],
                                                 false, st));
  return SENSE_OK;
}

extern "C" int sense_batch_cg_solve(sense_batch B, const float* const* s, float* const* x,
                                    const sense_cg_opts* opts, sense_cg_info* info,
                                    void* stream) {
  BTRY(check_batch(B));
  if (!s || !x || !opts) return set_error(SENSE_EINVAL, "null s, x or opts");
  if (opts->max_iter < 0 || !(opts->rel_tol >= 0.0))
    return set_error(SENSE_EINVAL, "max_iter and rel_tol must be >= 0");
  if (opts->refine_every != 0)
    return set_error(SENSE_EINVAL, "batched solves do not support residual replacement");
  if (opts->use_x0)
    return set_error(SENSE_EINVAL, "batched solves start from rho = 0 (use_x0 must be 0)");
  if (opts->prec != SENSE_PREC_TC_FP16 && opts->prec != SENSE_PREC_TC_SPLIT)
    return set_error(SENSE_EINVAL, "batched solves run on the tensor cores (TC_FP16, TC_SPLIT)");
  const int n = (int)B->plans.size();
  for (int b = 0; b < n; ++b)
    if (!s[b] || !x[b] || !is_device_pointer(s[b]) || !is_device_pointer(x[b]))
      return set_error(SENSE_EINVAL, "batched s and x must be device pointers");
  cudaStream_t st = (cudaStream_t)stream;
  for (int b = 0; b < n; ++b) BTRY(cg_begin(B->plans[b], (const float2*)s[b], opts, nullptr, st));
  const int N = opts->max_iter;
  if (N > 0) {
    // the first iteration runs directly (it also performs every one-time kernel set-up);
    // the others replay one captured iteration
    BTRY(batch_cg_iteration(B, opts->prec, st));
    if (N > 1 && (!B->gexec || B->graph_prec != opts->prec)) {
      if (B->gexec) cudaGraphExecDestroy(B->gexec);
      B->gexec = nullptr;
      cudaStream_t cs;
      SENSE_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaGraph_t g = nullptr;
      int rc = SENSE_OK;
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        rc = cuda_error(cudaGetLastError(), "cudaStreamBeginCapture");
      } else {
        rc = batch_cg_iteration(B, opts->prec, cs);
        const cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (rc == SENSE_OK && e != cudaSuccess) rc = cuda_error(e, "cudaStreamEndCapture");
      }
      if (rc == SENSE_OK && cudaGraphInstantiate(&B->gexec, g, 0) != cudaSuccess) {
        rc = cuda_error(cudaGetLastError(), "cudaGraphInstantiate");
        B->gexec = nullptr;
      }
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(cs);
      if (rc != SENSE_OK) return rc;
      B->graph_prec = opts->prec;
    }
    for (int it = 1; it < N; ++it) {
      NvtxRange nvtx("sense batch CG iteration (graph)");
      SENSE_CUDA_TRY(cudaGraphLaunch(B->gexec, st));
    }
  }
  for (int b = 0; b < n; ++b)
    BTRY(scatter_image(B->plans[b], B->plans[b]->vx, (float2*)x[b], opts->apply_j != 0, st));
  if (info)
    for (int b = 0; b < n; ++b) BTRY(cg_read_info(B->plans[b], &info[b], nullptr, st));
  if (info) return check_err(B);
  return SENSE_OK;
}

extern "C" int sense_batch_set_tuning(sense_batch B, int32_t chunk, int32_t seg_len) {
  BTRY(check_batch(B));
  if (chunk < 1 || chunk > 4096 || seg_len < 1 || seg_len > 64)
    return set_error(SENSE_EINVAL, "chunk must be 1..4096 and seg_len 1..64");
  B->seg_len = seg_len;
  if (chunk != B->chunk) {
    SENSE_CUDA_TRY(cudaDeviceSynchronize());
    B->chunk = chunk;
    return build_layout(B);
  }
  if (B->gexec) cudaGraphExecDestroy(B->gexec);
  B->gexec = nullptr;
  B->graph_prec = -1;
  return SENSE_OK;
}

extern "C" int sense_batch_autotune(sense_batch B, int32_t prec, int32_t* chunk,
                                    int32_t* seg_len, double* ms) {
  BTRY(check_batch(B));
  if (prec != SENSE_PREC_TC_FP16 && prec != SENSE_PREC_TC_SPLIT)
    return set_error(SENSE_EINVAL, "autotuning covers the tensor-core modes");
  cudaStream_t st;
  SENSE_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<const float2*> p;
  std::vector<float2*> q;
  for (auto* P : B->plans) {
    SENSE_CUDA_TRY(cudaMemsetAsync(P->vm, 0, (size_t)P->Lp * 8, st));
    p.push_back(P->vm);
    q.push_back(P->vq);
  }
  double best = 1e300;
  int best_c = B->chunk, best_s = B->seg_len;
  int rc = SENSE_OK;
  for (int c : CHUNK_CANDIDATES) {
    for (int s : SEG_CANDIDATES) {
      if ((rc = sense_batch_set_tuning(B, c, s)) != SENSE_OK) break;
      if ((rc = batch_normal(B, prec, p, q, false, st)) != SENSE_OK) break;  // warm-up
      cudaEventRecord(e0, st);
      for (int r = 0; r < 2 && rc == SENSE_OK; ++r) rc = batch_normal(B, prec, p, q, false, st);
      cudaEventRecord(e1, st);
      if (rc != SENSE_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = cuda_error(cudaGetLastError(), "autotune timing");
        break;
      }
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (t / 2 < best) {
        best = t / 2;
        best_c = c;
        best_s = s;
      }
    }
    if (rc != SENSE_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (rc != SENSE_OK) return rc;
  BTRY(check_err(B));
  BTRY(sense_batch_set_tuning(B, best_c, best_s));
  if (chunk) *chunk = best_c;
  if (seg_len) *seg_len = best_s;
  if (ms) *ms = best;
  return SENSE_OK;
}
