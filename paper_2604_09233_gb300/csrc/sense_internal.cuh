// Internal declarations shared by the translation units of libsense.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sense.h"

namespace sense {

// Named NVTX range for the host-side span of a scope (plan creation, a CG solve and each of
// its iterations, an E^H E apply, a tensor-core pass); visible to nsys / ncu --nvtx, a few
// tens of nanoseconds per range otherwise.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Anchor block size: samples are grouped in blocks of TILE consecutive samples, voxels
// in spatially compact blocks of TILE (k-d order). Every kernel tile lies inside one
// sample block and one voxel block along each of its two dimensions.
constexpr int TILE = 128;
constexpr int MAX_RP = 20;   // max basis rows kept in the FP32 bilinear part
constexpr int MAX_CP = 64;   // max (padded) coils
// Streamed-side image bytes that one stream-K chunk of the tensor-core passes may span: a
// quarter of the 126 MB L2, so that the CTAs (which drift apart by part of a chunk) find the
// images of the chunk they share in L2 instead of re-reading them from HBM.
constexpr long long TC_L2_CHUNK_BYTES = 32ll << 20;

// Device scalars of the CG recurrence (double), indices into plan->scal.
enum ScalarSlot {
  SC_RR = 0,       // r^H r of the current residual
  SC_RR0,          // r_0^H r_0
  SC_PQ_RE,        // p^H q
  SC_PQ_IM,
  SC_A_RE,         // alpha / beta of the listing (the step length)
  SC_A_IM,
  SC_B_RE,         // ratio for the p update
  SC_B_IM,
  SC_SS,           // ||s||^2
  SC_STOP,         // 0 running, 1 converged (tol), 2 breakdown, 3 non-finite
  SC_ITER,         // iterations completed
  SC_TOL2,         // rel_tol^2 * rr0 (0 disables)
  SC_MAXIT,        // N_It
  SC_RR_PREV,      // r^H r of the previous iteration (for a replaced residual)
  SC_COUNT
};

struct Workspace {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace sense

struct sense_plan_s {
  int device = 0;
  int num_sms = 0;
  int64_t L = 0, K = 0;
  int C = 0, P1 = 0;
  int64_t Lp = 0, Kp = 0;  // padded to TILE
  int Cp = 0;              // padded to 8/16/32/64
  int nsb = 0, nvb = 0;    // sample / voxel blocks
  int r = 0, RP = 0;       // rows kept in the bilinear part, padded to a multiple of 4
  std::vector<int> rows;   // which rows of K R vary inside blocks

  // host master geometry
  std::vector<double> Kh;      // [K][P1]
  std::vector<double> Rh;      // [P1][L] user order
  std::vector<float> Sh;       // [L][C] complex interleaved
  std::vector<float> jh;       // [L] (ones if absent)
  bool has_j = false;
  std::vector<int32_t> perm;   // [Lp] plan slot -> user voxel (-1 = padding)

  // device geometry
  double* dKd = nullptr;     // [Kp][P1]  K / 2pi (turns per unit of R), pad rows = centre
  double* dRd = nullptr;     // [P1][Lp]  R in plan order, pad = centre
  double* dKc = nullptr;     // [nsb][P1] sample-block centres (turn units)
  double* dRc = nullptr;     // [nvb][P1] voxel-block centres
  int* drows = nullptr;      // [r]
  int32_t* dperm = nullptr;  // [Lp]
  float* dK = nullptr;       // [Kp][RP]  (K/2pi - Kc) on kept rows
  float* dR = nullptr;       // [Lp][RP]  (R - Rc) on kept rows
  int RT = 0;                // kept rows padded to the tensor-core kernels' row count
  float* dKt = nullptr;      // [nsb][RT][TILE] the same deltas, row-major per block
  float* dRt = nullptr;      // [nvb][RT][TILE]
  float* Aanc = nullptr;     // [nsb][Lp] frac(Kc . R(l))
  float* Banc = nullptr;     // [nvb][Kp] frac((K(k) - Kc) . Rc)
  float* AancR = nullptr;    // the same two tables in radians, 2 pi frac(.)
  float* BancR = nullptr;
  // tensor-core phase operands (FP16 hi/lo images of the kept rows of dK and dR, scaled)
  int nkp = 1;               // K-steps of 16 rows: 1 (RT <= 16) or 2
  float ph_unscale = 1.0f;
  uint8_t* phK_row = nullptr;  // [nsb][TCP_ROW_BYTES] samples as rows (E pass)
  uint8_t* phR_row = nullptr;  // [nvb][TCP_ROW_BYTES] voxels as rows (E^H pass)
  uint8_t* phR_col = nullptr;  // [nvb][tcp_col_bytes] voxels streamed (E pass)
  uint8_t* phK_col = nullptr;  // [nsb][tcp_col_bytes] samples streamed (E^H pass)
  float2* S = nullptr;       // [Lp][Cp]  S o j, plan order
  float* jv = nullptr;       // [Lp] j in plan order (1 for padding)
  float* tk = nullptr;       // [Kp] K(:,0) = t_k as float (0 for padding)

  // FP32 path workspace
  int nsplit_e = 1, vb_per_split = 1;  // encode: voxel-block split
  int nsplit_a = 1, sb_per_split = 1;  // adjoint: sample-block split
  float2* Ypart = nullptr;   // [nsplit_e][Kp][Cp]
  float2* Y = nullptr;       // [Kp][Cp] operator scratch (E p inside E^H E)
  float2* Ydata = nullptr;   // [Kp][Cp] coil data Sigma in the internal layout (CG)
  float2* Xpart = nullptr;   // [nsplit_a][Lp]

  // CG vectors (plan order) and scalars
  float2 *vx = nullptr, *vr = nullptr, *vp = nullptr, *vq = nullptr, *vb = nullptr,
         *vm = nullptr;
  double* scal = nullptr;    // [SC_COUNT]
  double* hist = nullptr;    // [(max_hist)*3]
  int max_hist = 0;
  double* red = nullptr;     // reduction partials
  unsigned* counter = nullptr;
  int red_blocks = 0;

  // host staging (for host-pointer arguments)
  float2* stage_s = nullptr;   // [K][C] device staging for user-layout data
  float2* stage_m = nullptr;   // [L]    device staging for user-layout images

  // tensor-core path (sense_tc.cu)
  int tc_grid = 0;                 // persistent CTAs launched (<= pairs of blocks)
  int tc_grid_req = 0;             // requested CTAs (one per SM by default)
  int tc_seg_len = 0;              // drain the TMEM accumulators every this many pairs (0: by
                                   // precision, tc_seg_for)
  int tc_wait_us = 0;              // bounded-wait limit of the tensor-core kernels (0: ~2 s)
  long long tc_wait_cycles = 0;    // the same in SM clock cycles (0: the kernel's default)
  int tc_test_hold = 0;            // time-out tests: stage CTA 0's loader withholds (+1)
  int clock_khz = 0;               // maximum SM clock (cudaDevAttrClockRate)
  int min_rt = 0;                  // lower bound on RT (uniform kernels across a batch)
  int64_t geom_version = 0;        // incremented whenever the geometry arrays are rebuilt
  int tc_slots_e = 1, tc_slots_a = 1;
  // stream-K slot tables of E / E^H: slot of (chunk c, row block o, CTA i) =
  // slot_base[c * n_outer + o] + i; partial slots per row block
  int *tc_first_e = nullptr, *tc_nslot_e = nullptr;  // [chunks_e][nsb], [nsb]
  int *tc_first_a = nullptr, *tc_nslot_a = nullptr;  // [chunks_a][nvb], [nvb]
  int tc_chunk_e = 1, tc_chunk_a = 1;              // streamed blocks per chunk
  int tc_inner_chunk = 0;                          // forced chunk width (0: automatic)
  uint8_t* Qimg = nullptr;         // B image of S o p   [nvb][2][2][2Cp][128 B]
  uint8_t* Yimg = nullptr;         // B image of Sigma   [nsb][2][2][2Cp][128 B]
  float *qscale = nullptr, *yscale = nullptr;  // [Cp] per-coil unscale factors
  unsigned* colmax = nullptr;      // [2][Cp] per-coil maxima (float bits)
  float2* Ypart_tc = nullptr;      // [tc_slots_e][Kp][Cp]
  float2* Xpart_tc = nullptr;      // [tc_slots_a][Lp][tc_xpart_coils]
  int* tc_err = nullptr;           // time-out word written by the tensor-core kernels
  uint4* p_enc = nullptr;          // stored-P mode: phase tiles of the E pass
  uint4* p_adj = nullptr;          // and of the E^H pass (conjugated, transposed)

  // gradient workspace (sense_grad.cu), allocated on first use
  float2* Yg = nullptr;            // [Kp][Cp] E of an adjoint vector
  float2* Yt = nullptr;            // [Kp][Cp] t-weighted data
  float2* vt = nullptr;            // [Lp] E^H (t o y)
  float* gw = nullptr;             // [Lp] d/d omega accumulator, plan order
  float2 *gx = nullptr, *gr = nullptr, *gp = nullptr, *gq = nullptr;  // [Lp] CG adjoints
  double* gsc = nullptr;           // [8] backward scalars
  int seg_cap = 0;                 // iterations the segment store holds
  float2 *seg_p = nullptr, *seg_q = nullptr, *seg_r = nullptr;  // [seg_cap][Lp]
  float2* seg_Y = nullptr;         // [seg_cap][Kp][Cp]  E p_n
  double* seg_sc = nullptr;        // [seg_cap][SC_COUNT]

  // diagnostics (sense_diag.cu)
  int64_t n_launch = 0;
  bool prof_on = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_events;
  size_t prof_used = 0;
};

namespace sense {

// plan creation with lower bounds on the padded coil count and the delta rows (0 = none)
int plan_create(const sense_problem* prob, int min_cp, int min_rt, sense_plan_s** out);

// error reporting -------------------------------------------------------------------
int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* what);
#define SENSE_CUDA_TRY(expr)                                   \
  do {                                                         \
    cudaError_t _e = (expr);                                   \
    if (_e != cudaSuccess) return sense::cuda_error(_e, #expr); \
  } while (0)

bool is_device_pointer(const void* p);

// FP32 CUDA-core operator (sense_fp32.cu) --------------------------------------------
// All vectors in plan order / internal layouts. The stop flag (nullable) makes the
// kernels return immediately when nonzero (used inside a converged CG loop).
int fp32_encode_partials(sense_plan_s* P, const float2* m_plan, const double* stop,
                         cudaStream_t st);  // -> P->Ypart
int reduce_y(sense_plan_s* P, float2* Y_int, float2* s_user, const double* stop,
             cudaStream_t st);             // Ypart -> Y_int [Kp][Cp] and/or s_user [K][C]
int fp32_adjoint_partials(sense_plan_s* P, const float2* Y_int, const double* stop,
                          cudaStream_t st);  // -> P->Xpart

// vector kernels (sense_vec.cu) -------------------------------------------------------
int gather_image(sense_plan_s* P, const float2* m_user, float2* m_plan, cudaStream_t st);
int scatter_xpart(sense_plan_s* P, float2* m_user, bool apply_j, cudaStream_t st);
int scatter_image(sense_plan_s* P, const float2* v_plan, float2* m_user, bool apply_j,
                  cudaStream_t st);
int load_data(sense_plan_s* P, const float2* s_user, float2* Y_int, cudaStream_t st);
int reduce_xpart(sense_plan_s* P, float2* q_plan, const double* stop, cudaStream_t st);

// tensor-core operator (sense_tc.cu) ----------------------------------------------------
int tc_setup(sense_plan_s* P);
void tc_free(sense_plan_s* P);
// E p for p in plan order: Y_int [Kp][Cp] and/or s_user [K][C]; want_colmax also records
// the per-coil maxima of the result for a following tc_adjoint(colmax_ready = true).
int tc_encode(sense_plan_s* P, int prec, const float2* p_plan, float2* Y_int, float2* s_user,
              bool want_colmax, const double* stop, cudaStream_t st);
int tc_adjoint(sense_plan_s* P, int prec, const float2* Y_int, float2* q, bool colmax_ready,
               const double* stop, cudaStream_t st);
int tc_check_error(sense_plan_s* P);
int tc_set_tuning(sense_plan_s* P, int seg_len, int grid, int inner_chunk);

// diagnostics (sense_diag.cu) ----------------------------------------------------------
enum KernelClass { KC_TC_ENC = 0, KC_TC_ADJ = 1, KC_F32_ENC = 2, KC_F32_ADJ = 3 };
// Bracket one launch of class kc with events on st when profiling is on; call
// prof_begin before and prof_end after the launch.
int prof_begin(sense_plan_s* P, int kc, cudaStream_t st);
int prof_end(sense_plan_s* P, cudaStream_t st);
void prof_free(sense_plan_s* P);
inline void count_launch(sense_plan_s* P, int n = 1) { P->n_launch += n; }

// CG (sense_cg.cu) --------------------------------------------------------------------
// Host-pointer arguments are staged through plan buffers: inputs copied in before the work,
// outputs copied back (synchronously) after it.
struct Staged {
  const void* user;
  void* dev;
  bool host;
};
int stage_in(const void* user, void* buf, size_t bytes, cudaStream_t st, Staged* s);
Staged stage_out(void* user, void* buf);
int finish_out(const Staged& s, size_t bytes, cudaStream_t st);
int check_plan(sense_plan_s* P);
int check_prec(int prec);
int grid_for(sense_plan_s* P, int64_t n);
// One CG solve; with ckpt_every > 0 the state (r, p, scalars) before every ckpt_every-th
// iteration and the final scalars are written to ckpt (layout of sense_grad.cu); with
// iterates, every x_n (n = 0..max_iter, user order) to iterates[n].
int cg_run(sense_plan_s* P, const float* s, float* x, const sense_cg_opts* opts,
           double* history, sense_cg_info* info, int ckpt_every, uint8_t* ckpt,
           float2* iterates, cudaStream_t st);
int cg_begin(sense_plan_s* P, const float2* s_dev, const sense_cg_opts* opts, double* hist,
             cudaStream_t st, const float2* x0 = nullptr);
int cg_read_info(sense_plan_s* P, sense_cg_info* info, int* iters, cudaStream_t st);
int encode_internal(sense_plan_s* P, int prec, const float2* p_plan, float2* Y_int,
                    cudaStream_t st);
int cg_step_alpha(sense_plan_s* P, cudaStream_t st);
int cg_step_update(sense_plan_s* P, double* hist, cudaStream_t st);
int cg_step_p(sense_plan_s* P, cudaStream_t st);
int apply_normal_internal(sense_plan_s* P, int prec, const float2* p_plan, float2* q_plan,
                          const double* stop, cudaStream_t st);
int adjoint_internal(sense_plan_s* P, int prec, const float2* Y_int, float2* q_plan,
                     const double* stop, cudaStream_t st);

// gradients and checkpoints (sense_grad.cu) ------------------------------------------------
void grad_free(sense_plan_s* P);
int ckpt_save(sense_plan_s* P, uint8_t* ckpt, int64_t slot, cudaStream_t st);
int ckpt_final(sense_plan_s* P, uint8_t* ckpt, cudaStream_t st);

}  // namespace sense
