// Tensor-core pass: the data the pass kernel reads and the host entry points shared by the
// single-problem operator (sense_tc.cu) and the batched solver (sense_batch.cu).
#pragma once
#include "sense_internal.cuh"

namespace sense {
namespace tc {

// One problem instance as the pass kernel sees it.
struct InstDesc {
  const float* rowT;     // [n_outer][RT][128] own-dimension deltas (dK for ENC, dR for ADJ)
  const float* colT;     // [n_inner][RT][128] streamed deltas
  const float* rowAnc;   // [n_inner][rows_total] (Banc for ENC, Aanc for ADJ)
  const float* colAnc;   // [n_outer][cols_total] (Aanc for ENC, Banc for ADJ)
  const uint8_t* Bimg;   // [n_inner][2 halves][NPART][2*CP rows][128 B]
  const float* bscale;   // [CP] 2^-e unscale per coil
  const float2* S;       // [rows_total][CP] (ADJ epilogue of the 64-coil kernel)
  float2* out;           // ENC: [slots][rows_total][CP]; ADJ: the same for the phase kernel,
                         // [slots][rows_total] (coils combined) for the 64-coil kernel
  const double* stop;    // CG stop flag of the instance (nullable; work queue only)
  long long rows_total, cols_total;
  int n_outer, n_inner;
  int chunk;             // work queue: streamed blocks per work item (slot = first / chunk)
  int pad;
  // stored phase tiles (stored-P mode): per (row block, streamed block) pair 16 chunks
  // (stage, warpgroup, half) of [4 matrices: re hi, re lo, im hi, im lo][128 rows][8 FP16]
  const uint4* stored;
  // tensor-core phase (sense_tcp.cu): FP16 hi/lo operand images of the local bilinear phase,
  // 128B-swizzled K-major: the row side [n_outer][128 rows][128 B] in natural order and the
  // streamed side [n_inner][TCP_COL_BYTES] in the permuted stage order; anchors in radians.
  const uint8_t* rowPh;
  const uint8_t* colPh;
  const float* rowAncR;  // [n_inner][rows_total] radians
  const float* colAncR;  // [n_outer][cols_total] radians
  float ph_unscale;      // the phase images' products are radians times 1 / ph_unscale
  int pad2;
};

// Two schedules feed the same kernel:
//   stream-K (one instance, inst == nullptr): the streamed blocks are cut into chunks of
//     `chunk_inner` (one chunk unless the streamed-side images of all blocks exceed an L2
//     budget); chunk by chunk, CTA i takes the pairs [iW/G, (i+1)W/G) of the chunk's
//     flattened (row block, streamed block) space, so all CTAs read the same chunk's images
//     at about the same time; the partial slot of (chunk c, row block o) is
//     first_cta[c * n_outer + o] + i;
//   work queue (inst != nullptr): CTAs claim items {instance, row block, first, end streamed
//     block} with an atomic counter (zeroed before the launch), skipping stopped instances;
//     an item is one run and its slot is first / chunk.
struct Params {
  InstDesc d0;           // the instance of the stream-K schedule
  const InstDesc* inst;  // work queue: per-instance descriptors
  const int4* items;     // work queue: [n_items]
  unsigned* next;        // work queue: claim counter
  int n_items;
  const int* first_cta;  // stream-K: slot base [chunks][n_outer] (slot = base + CTA index)
  int chunk_inner;       // stream-K: streamed blocks per chunk (n_inner: one chunk)
  long long W;           // stream-K: n_outer * n_inner
  int* err;              // device error word (nonzero after a time-out)
  const double* stop;    // stream-K: CG stop flag (nullable)
  int seg_len;           // accumulator drain interval (pairs of 128 x 128)
  long long wait_limit;  // bounded waits give up after this many SM cycles (0: ~2 s)
  int hold;              // tests only: > 0 makes CTA 0's loader withhold stage hold - 1
  uint4* emit;           // tensor-core phase kernel, stream-K, split: also write the FP16
                         // tiles it generates in the stored-P layout (nullable)
};

// Per-stage metadata passed from the loader to the MMA and generator warps.
struct Meta {
  int inst, o, in, flags;  // flags: bit 0 first pair of a run, bit 1 last pair, bit 2 end
  int slot, pad0, pad1, pad2;
};
constexpr int META_FIRST = 1, META_LAST = 2, META_END = 4;

enum Mode { ENC = 0, ADJ = 1 };

}  // namespace tc

// Launch one pass (template chosen by npart, cp = padded coils, rt = delta rows) on G CTAs;
// stored: the phase tiles come from prm's descriptors' `stored` arrays. Up to 32 padded
// coils the generated passes run the tensor-core phase kernel (sense_tcp.cu).
int tc_launch(sense_plan_s* P, int mode, int npart, int cp, int rt, const tc::Params& prm, int G,
              cudaStream_t st, bool stored = false);
namespace tc {
// Tensor-core phase kernel (sense_tcp.cu): streamed-side image bytes per block for nkp
// K-steps of 16 phase rows (nkp = 0: the stored-P variant, which reads its tiles from HBM),
// the row-side bytes, whether it serves a launch, and the launch.
constexpr int tcp_col_bytes(int nkp) { return nkp == 0 ? 0 : nkp == 1 ? 8192 : 16384; }
constexpr int TCP_ROW_BYTES = 16384;
bool tcp_covers(int cp, bool stored);
int tcp_launch(sense_plan_s* P, int mode, int npart, int cp, int nkp, const Params& prm, int G,
               cudaStream_t st);
}  // namespace tc
// Stored-P mode: generate (enable) or free the phase tiles of both passes.
int tc_store_p(sense_plan_s* P, bool enable, cudaStream_t st);
// B image of src (Y_int layout, nrows x Cp) or of S o pv; colmax computed unless have_colmax.
int tc_make_image(sense_plan_s* P, int npart, const float2* src, const float2* pv,
                  long long nrows, unsigned* colmax, float* bscale, uint8_t* img,
                  bool have_colmax, cudaStream_t st);
// Sum of partial slots: Y_int / s_user (+ colmax) from Ypart [slots][Kp][Cp] with nslot per
// sample block; q from Xpart [slots][Lp] with nslot per voxel block.
int tc_reduce_y(sense_plan_s* P, const float2* Ypart, const int* nslot, float2* Y_int,
                float2* s_user, unsigned* colmax, const double* stop, cudaStream_t st);
// Values per partial row of the E^H pass: Cp (the phase kernel writes per-coil rows; the coil
// combine happens in tc_reduce_x) or 1 (the 64-coil kernel combines the coils itself).
int tc_xpart_coils(const sense_plan_s* P);
int tc_reduce_x(sense_plan_s* P, const float2* Xpart, const int* nslot, float2* q,
                const double* stop, cudaStream_t st);

}  // namespace sense
