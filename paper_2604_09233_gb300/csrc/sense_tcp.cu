// Tensor-core (tcgen05) E and E^H in which the phase of every (sample, voxel) pair is also
// formed on the tensor cores.
//
// A pass contracts the phase matrix P = e^{i K R} (Eq. 4) against a thin complex operand over
// one of its dimensions, as in sense_tc.cu:
//   ENC (s = E m, Eq. 4):    rows = samples, streamed = voxels,  B = Q = S o m
//   ADJ (m = E^H s, Eq. 5):  rows = voxels,  streamed = samples, B = Sigma, conjugate tile
// With block anchors A, B (FP64, reduced mod 2 pi) the phase of a pair is
//   phi(k, l) = A(b(k), l) + B(v(l), k) + D(k, l),  D = 2 pi sum_q dK(k, q) dR(l, q),
// and D, the local bilinear part, is a small GEMM with K = the kept basis rows (<= 32). Here
// it runs on the tensor cores as three FP16 products of hi/lo splits (hi hi + hi lo + lo hi,
// FP32 accumulation) of prebuilt operand images, once per 128 x 64 stage, into the tensor
// memory slot where that stage's exponential tile is written next. The generator warps then
// read the phases back, add the anchors, evaluate cos/sin on the special function unit,
// split into FP16 hi (+ lo) and write the tile over the phases; the MMA warp contracts it
// with the B operand as before. The E^H pass writes the tile of e^{+i phi} and takes the
// conjugate in the accumulator read-out.
// Per CTA (one per SM, persistent, 20 warps):
//   16 generator warps  : phases out of TMEM -> anchors -> sin/cos -> FP16 tile into TMEM (for
//                         single tiles in two groups of 8 on alternating stages); at segment
//                         ends they drain the accumulators into running sums, and at run ends
//                         write the run's rows per coil (both passes; the E^H pass's coil
//                         combine with S is done by the slot reduction);
//   1 phase warp        : the phase MMAs of the stages ahead (A and B in shared memory), each
//                         into the TMEM slot of its stage once that slot's contraction is done;
//   2 contraction warps : the contraction MMAs of each stage (A in TMEM, B in shared memory),
//                         one warp per accumulator (the tile's real and imaginary parts);
//   1 loader warp       : bulk copies of the B image, the streamed phase operand, the anchors
//                         of every streamed block and the row phase operand of every run,
//                         and the shared-memory metadata ring of the schedule.
// Schedules: stream-K for one problem (two-level when the streamed-side images exceed an L2
// budget), a work queue for a batch. Every wait is bounded.
#include <cuda_fp16.h>

#include <algorithm>

#include "sense_ptx.cuh"
#include "sense_tc.cuh"

namespace sense {
namespace tcp {

using namespace sense::tc;

constexpr int NGEN_WARPS = 16;
constexpr int MMA_WARP = 16;    // issues the D1 contraction MMAs
constexpr int LOAD_WARP = 17;
constexpr int MMA2_WARP = 18;   // issues the D2 contraction MMAs
constexpr int PHASE_WARP = 19;  // issues the phase MMAs
constexpr int NTHREADS = 20 * 32;
constexpr uint32_t TMEM_COLS = 512;

template <int CP, int NPART, int NKP>
struct Lay {
  static constexpr int BROWS = 2 * CP;
  static constexpr int B_HALF = NPART * BROWS * 128;  // B image of one 64-wide stage
  static constexpr int B_BYTES = 2 * B_HALF;           // one streamed block
  static constexpr int PC_BYTES = tcp_col_bytes(NKP);  // streamed phase operand, one block
  static constexpr int PR_BYTES = TCP_ROW_BYTES;       // row phase operand, one row block
  // MMA width N = 2 CP (the rows [B_re; B_im] of one part of the B image); the accumulators
  // D1 (the tile's real part times B) and D2 (its imaginary part) are N columns each.
  static constexpr int NMMA = 2 * CP;
  // TMEM: accumulators D1, D2 in columns [0, 2 NMMA); tile slots (NPART x {re, im} FP16
  // matrices of 32 columns; the stage's FP32 phases occupy the slot's first 64 columns
  // until the tile is written over them) from ACOL0 to the end of the 512.
  static constexpr uint32_t ACOL0 = 2 * NMMA > 128 ? 2 * NMMA : 128;
  static constexpr int SLOT_COLS = NPART * 64;
  static constexpr int NSLOT_FIT = (int)((512 - ACOL0) / SLOT_COLS);
  static constexpr int NSLOT = NSLOT_FIT > 4 ? 4 : NSLOT_FIT;
  static constexpr int NBUF = 3;
};

template <int CP, int NPART, int NKP>
constexpr size_t smem_bytes() {
  using LY = Lay<CP, NPART, NKP>;
  return 1024 + LY::NBUF * (LY::B_BYTES + LY::PC_BYTES) + 2 * LY::PR_BYTES +
         2 * LY::NBUF * 128 * 4 + (CP / 4) * NGEN_WARPS * 32 * 8 +
         LY::NBUF * sizeof(Meta) + 40 * 8 + 16;
}

// EMIT: also write every generated tile to Params::emit (the pass that builds the stored-P
// tiles); the ordinary passes are compiled without that code.
template <int MODE, int CP, int NPART, int NKP, bool EMIT>
__global__ void __launch_bounds__(NTHREADS, 1) tcp_pass_kernel(Params p) {
  using LY = Lay<CP, NPART, NKP>;
  constexpr int NBUF = LY::NBUF;
  constexpr int NSLOT = LY::NSLOT;
  constexpr int CW = CP / 4;  // coils per warpgroup in the drains and the run output
  // NKP = 0: stored-P variant: the tiles are read from HBM (written by a generating pass with
  // Params::emit), no phase operands or anchors are loaded and no phase MMAs run
  constexpr bool STORED = NKP == 0;
  // generator groups on alternating stages: two for single tiles, one for split tiles
  constexpr int GROUPS = NPART == 1 ? 2 : 1;
  constexpr int GEN_PER_STAGE = NGEN_WARPS / GROUPS;  // generator warps that write a stage
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* sB = base;                                     // [NBUF][B_BYTES]
  uint8_t* sPc = sB + NBUF * LY::B_BYTES;                 // [NBUF][PC_BYTES]
  uint8_t* sPr = sPc + NBUF * LY::PC_BYTES;               // [2][PR_BYTES]
  float* sAnc = (float*)(sPr + 2 * LY::PR_BYTES);         // [NBUF][128] streamed anchors
  float* sRowAnc = sAnc + NBUF * 128;                     // [NBUF][128] row anchors
  float2* sRacc = (float2*)(sRowAnc + NBUF * 128);        // [CP/4][512] running sums
  Meta* sMeta = (Meta*)(sRacc + CW * NGEN_WARPS * 32);    // [NBUF]
  uint64_t* bars = (uint64_t*)(sMeta + NBUF);
  uint64_t* full = bars;                 // [NBUF] streamed block landed
  uint64_t* empty = full + NBUF;         // [NBUF] streamed block consumed
  uint64_t* rfull = empty + NBUF;        // [2] row phase operand landed
  uint64_t* rempty = rfull + 2;          // [2] row phase operand no longer read
  uint64_t* pfull = rempty + 2;          // [NSLOT] phases of the slot's stage in TMEM
  uint64_t* tfull = pfull + NSLOT;       // [NSLOT] tile written
  uint64_t* tempty = tfull + NSLOT;      // [NSLOT] contraction MMAs of the slot done
  uint64_t* afull = tempty + NSLOT;      // accumulator full
  uint64_t* aempty = afull + 1;          // accumulator drained
  uint64_t* drain = aempty + 1;          // [3] final MMA drain of each issuing warp
  uint32_t* tmem_slot = (uint32_t*)(drain + 3);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (p.stop && *p.stop != 0.0) return;
  const bool queue = p.inst != nullptr;
  auto desc = [&](int b) -> const InstDesc& { return queue ? p.inst[b] : p.d0; };

  const long long i = blockIdx.x;
  const int F = p.seg_len;
  const long long LIM = p.wait_limit > 0 ? p.wait_limit : WAIT_LIMIT_CYCLES;

  if (threadIdx.x == 0) {
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(smem_u32(&full[b]), 1);
      mbar_init(smem_u32(&empty[b]), NGEN_WARPS + 3);  // generators and the three issuers
    }
    for (int r = 0; r < 2; ++r) {
      mbar_init(smem_u32(&rfull[r]), 1);
      mbar_init(smem_u32(&rempty[r]), 1);
    }
    for (int s = 0; s < NSLOT; ++s) {
      mbar_init(smem_u32(&pfull[s]), 1);
      mbar_init(smem_u32(&tfull[s]), GEN_PER_STAGE);
      mbar_init(smem_u32(&tempty[s]), 2);
    }
    mbar_init(smem_u32(afull), 2);
    mbar_init(smem_u32(aempty), GEN_PER_STAGE);  // the drainers (group 0)
    for (int r = 0; r < 3; ++r) mbar_init(smem_u32(drain + r), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr int NM = LY::NMMA;
  const uint32_t D1 = tmem, D2 = tmem + NM;
  // Tensor memory is not cleared between kernels; the accumulator columns are zeroed before
  // the first MMA (warpgroup g zeroes columns [g NM / 2, (g+1) NM / 2) of its lane quarter).
  if (warp < NGEN_WARPS) {
    const uint32_t zr[4] = {0u, 0u, 0u, 0u};
    const uint32_t zb = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (warp >> 2) * (NM / 2);
#pragma unroll
    for (int c = 0; c < NM / 2; c += 4) tmem_st4(zb + c, zr);
    tmem_st_wait();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == LOAD_WARP) {
    // ------------------------------------------------------------------ loader
    if (lane == 0) {
      long long it = 0;   // blocks pushed
      Ring<NBUF> rb;      // ring position of block it
      int run = 0;  // runs started: run r's row phase operand goes to ring slot r & 1
      bool ok = true;
      auto push = [&](int b, int o, int in, int flags, int slot) -> bool {
        const int buf = rb.idx;
        if (it >= NBUF &&
            !mbar_wait(smem_u32(&empty[buf]), rb.phase ^ 1u, abort_flag, p.err, 1, LIM))
          return false;
        if (!STORED && !(flags & META_END) && (flags & META_FIRST)) {
          const int rs = run & 1;
          const uint32_t ru = (uint32_t)(run >> 1);
          if (ru > 0 &&
              !mbar_wait(smem_u32(&rempty[rs]), (ru - 1) & 1u, abort_flag, p.err, 11, LIM))
            return false;
          const uint32_t rb = smem_u32(&rfull[rs]);
          mbar_arrive_expect_tx(rb, LY::PR_BYTES);
          bulk_g2s(smem_u32(sPr + rs * LY::PR_BYTES),
                   desc(b).rowPh + (long long)o * LY::PR_BYTES, LY::PR_BYTES, rb);
          ++run;
        }
        Meta m;
        m.inst = b; m.o = o; m.in = in; m.flags = flags; m.slot = slot;
        m.pad0 = m.pad1 = m.pad2 = 0;
        sMeta[buf] = m;
        const uint32_t fb = smem_u32(&full[buf]);
        if (flags & META_END) {
          mbar_arrive(fb);
        } else if (p.hold > 0 && i == 0 && it == p.hold - 1) {
          // test of the time-out path: this block's arrival is never signalled and no copy
          // is issued for it, so every wait on it runs out after LIM cycles
        } else {
          const InstDesc& d = desc(b);
          mbar_arrive_expect_tx(fb, LY::B_BYTES + (STORED ? 0u : LY::PC_BYTES + 1024u));
          bulk_g2s(smem_u32(sB + buf * LY::B_BYTES), d.Bimg + (long long)in * LY::B_BYTES,
                   LY::B_BYTES, fb);
          if (!STORED) {
            bulk_g2s(smem_u32(sPc + buf * LY::PC_BYTES),
                     d.colPh + (long long)in * LY::PC_BYTES, LY::PC_BYTES, fb);
            bulk_g2s(smem_u32(sAnc + buf * 128),
                     d.colAncR + (long long)o * d.cols_total + (long long)in * 128, 512u, fb);
            bulk_g2s(smem_u32(sRowAnc + buf * 128),
                     d.rowAncR + (long long)in * d.rows_total + (long long)o * 128, 512u, fb);
          }
        }
        ++it;
        rb.next();
        return true;
      };
      if (!queue) {
        // chunk by chunk of streamed blocks, this CTA's share of the chunk's pairs
        const long long G = gridDim.x;
        const int n_inner = p.d0.n_inner, n_outer = p.d0.n_outer;
        const int CH = p.chunk_inner > 0 ? p.chunk_inner : n_inner;
        for (int c0 = 0, c = 0; c0 < n_inner && ok; c0 += CH, ++c) {
          const int wc = min(CH, n_inner - c0);
          const long long Wc = (long long)n_outer * wc;
          const long long w0 = i * Wc / G, w1 = (i + 1) * Wc / G;
          int o = (int)(w0 / wc), in = (int)(w0 % wc);
          for (long long w = w0; w < w1 && ok; ++w) {
            const int flags = ((w == w0 || in == 0) ? META_FIRST : 0) |
                              ((w + 1 == w1 || in + 1 == wc) ? META_LAST : 0);
            ok = push(0, o, c0 + in, flags, p.first_cta[(long long)c * n_outer + o] + (int)i);
            if (++in == wc) {
              in = 0;
              ++o;
            }
          }
        }
      } else {
        while (ok) {
          const unsigned k = atomicAdd(p.next, 1u);
          if (k >= (unsigned)p.n_items) break;
          const int4 itm = p.items[k];
          const InstDesc& d = desc(itm.x);
          if (d.stop && *(volatile const double*)d.stop != 0.0) continue;
          const int slot = itm.z / d.chunk;
          for (int in = itm.z; in < itm.w && ok; ++in)
            ok = push(itm.x, itm.y, in,
                      (in == itm.z ? META_FIRST : 0) | (in + 1 == itm.w ? META_LAST : 0), slot);
        }
      }
      if (ok) ok = push(0, 0, 0, META_END, 0);
      // wait for the copies this warp issued (the last NBUF blocks and the row operands of
      // the last two runs) before the CTA can exit
      const long long n = it;
      for (long long k = (n > NBUF ? n - NBUF : 0); k < n; ++k) {
        const int buf = (int)(k % NBUF);
        const long long t0 = clock64();
        while (!mbar_try_wait(smem_u32(&full[buf]), (uint32_t)(k / NBUF) & 1u)) {
          if (clock64() - t0 > LIM) {
            atomicCAS(p.err, 0, 9);
            break;
          }
        }
      }
      for (int r = (run > 2 ? run - 2 : 0); r < run; ++r) {
        const long long t0 = clock64();
        while (!mbar_try_wait(smem_u32(&rfull[r & 1]), (uint32_t)(r >> 1) & 1u)) {
          if (clock64() - t0 > LIM) {
            atomicCAS(p.err, 0, 14);
            break;
          }
        }
      }
    }
  } else if (warp == PHASE_WARP) {
    // ------------------------------------------------------------------ phase MMAs
    // D(stage) = A_ph B_ph^T into the stage's tile slot, as soon as the slot's previous
    // contraction MMAs are done and the operands have landed; it runs ahead of the
    // generators by up to NSLOT stages.
    if (lane == 0) {
      constexpr uint32_t idesc_ph = idesc_f16(64);
      bool ok = true;
      Ring<NBUF> rb;
      Ring<NSLOT> rs;
      int warm = 0;  // stages issued, counted up to NSLOT (a slot's first use has no wait)
      int prun = 0, prs = 0;
      for (; ok; rb.next()) {
        const int buf = rb.idx;
        if (!mbar_wait(smem_u32(&full[buf]), rb.phase, abort_flag, p.err, 2, LIM)) {
          ok = false;
          break;
        }
        const int flags = sMeta[buf].flags;
        if (flags & META_END) break;
        if (!STORED && (flags & META_FIRST)) {
          prs = prun & 1;
          if (!mbar_wait(smem_u32(&rfull[prs]), (uint32_t)(prun >> 1) & 1u, abort_flag, p.err,
                         12, LIM)) {
            ok = false;
            break;
          }
          ++prun;
        }
        // descriptors of the row operand (this run) and of the block's streamed operand; a
        // 32-byte step inside a 128-byte row adds 2 to the start-address field
        const uint64_t da = desc_sw128(smem_u32(sPr + prs * LY::PR_BYTES));
        const uint64_t db0 = desc_sw128(smem_u32(sPc + buf * LY::PC_BYTES));
        for (int st = 0; st < 2; ++st, rs.next()) {
          const int slot = rs.idx;
          // the slot is free once the contraction MMAs of its previous stage have completed
          if (warm < NSLOT) {
            ++warm;
          } else if (!mbar_wait(smem_u32(&tempty[slot]), rs.phase ^ 1u, abort_flag, p.err, 13,
                                LIM)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dcol = tmem + LY::ACOL0 + slot * LY::SLOT_COLS;
          const uint64_t db = db0 + (uint64_t)(NKP == 1 ? 4 * st : 512 * st);
          // hi hi, hi lo, lo hi over the NKP K-steps (stored variant: no MMA; the commit then
          // only tells the generators that the slot is free)
#pragma unroll
          for (int term = 0; term < (STORED ? 0 : 3); ++term) {
            const int pa = term == 2 ? 1 : 0, pb = term == 1 ? 1 : 0;
#pragma unroll
            for (int k = 0; k < NKP; ++k)
              mma_ss(dcol, da + (uint64_t)(2 * (pa * NKP + k)), db + (uint64_t)(2 * (pb * NKP + k)),
                     idesc_ph, (term == 0 && k == 0) ? 0u : 1u);
          }
          tc_commit(smem_u32(&pfull[slot]));
        }
        if (!ok) break;
        // the block's streamed operand, and at a run's end its row operand, are read
        tc_commit(smem_u32(&empty[buf]));
        if (!STORED && (flags & META_LAST)) tc_commit(smem_u32(&rempty[prs]));
      }
      (void)ok;
      tc_commit(smem_u32(drain + 2));
      const long long t0 = clock64();
      while (!mbar_try_wait(smem_u32(drain + 2), 0u)) {
        if (clock64() - t0 > LIM) {
          atomicCAS(p.err, 0, 10);
          break;
        }
      }
    }
  } else if (warp == MMA_WARP || warp == MMA2_WARP) {
    // ------------------------------------------------------------------ contraction MMAs
    // Two threads issue, each into its own accumulator (role 0: D1 = A_re B^T, role 1: D2 =
    // A_im B^T): one tcgen05.mma takes a thread several tens of cycles to issue, and these
    // MMAs are thin (N = 2 CP).
    const int role = warp == MMA_WARP ? 0 : 1;
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(NM);
      const uint32_t dst = role == 0 ? D1 : D2;
      bool ok = true;
      Ring<NBUF> rb;
      Ring<NSLOT> rs;
      int seg = 0, seg_pos = 0;  // segments issued; position of the block in its segment
      for (; ok; rb.next()) {
        const int buf = rb.idx;
        if (!mbar_wait(smem_u32(&full[buf]), rb.phase, abort_flag, p.err, 15, LIM)) {
          ok = false;
          break;
        }
        const int flags = sMeta[buf].flags;
        if (flags & META_END) break;
        if (flags & META_FIRST) seg_pos = 0;
        const bool seg_first = seg_pos == 0;
        const bool seg_last = (flags & META_LAST) || seg_pos + 1 == F;
        seg_pos = seg_last ? 0 : seg_pos + 1;
        if (seg_first && seg > 0) {
          if (!mbar_wait(smem_u32(aempty), (uint32_t)(seg - 1) & 1u, abort_flag, p.err, 3, LIM)) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        const uint32_t sbuf = smem_u32(sB + buf * LY::B_BYTES);
        for (int st = 0; st < 2; ++st, rs.next()) {
          const int slot = rs.idx;
          if (!mbar_wait(smem_u32(&tfull[slot]), rs.phase, abort_flag, p.err, 4, LIM)) {
            ok = false;
            break;
          }
          tc_fence_after();
          // this role's tile part (real or imaginary) in the slot: hi at +0, lo at +32
          const uint32_t am = tmem + LY::ACOL0 + slot * LY::SLOT_COLS + (uint32_t)(role * 32 * NPART);
          const uint64_t dh = desc_sw128(sbuf + st * LY::B_HALF);
          const uint64_t dl = dh + (uint64_t)((2 * CP * 128) >> 4);   // the B image's lo rows
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t acc = (seg_first && st == 0 && k == 0) ? 0u : 1u;
            const uint64_t kh = dh + (uint64_t)(2 * k);
            // D += A_hi B_hi (+ A_hi B_lo + A_lo B_hi)
            mma_ts(dst, am + 8 * k, kh, idesc, acc);
            if (NPART == 2) {
              mma_ts(dst, am + 8 * k, dl + (uint64_t)(2 * k), idesc, 1u);
              mma_ts(dst, am + 32 + 8 * k, kh, idesc, 1u);
            }
          }
          tc_commit(smem_u32(&tempty[slot]));
        }
        if (!ok) break;
        tc_commit(smem_u32(&empty[buf]));
        if (seg_last) {
          tc_commit(smem_u32(afull));
          ++seg;
        }
      }
      (void)ok;
      // drain every MMA issued before the accumulators / TMEM go away
      tc_commit(smem_u32(drain + role));
      const long long t0 = clock64();
      while (!mbar_try_wait(smem_u32(drain + role), 0u)) {
        if (clock64() - t0 > LIM) {
          atomicCAS(p.err, 0, 10);
          break;
        }
      }
    }
  } else {
    // ------------------------------------------------------------------ generators
    // Split tiles: all 16 warps generate every stage; warp w covers the 32 rows of its TMEM
    // lane quarter (w & 3) and K-step w >> 2 (16 elements) of the stage's 64. Single tiles:
    // two groups of 8 warps on alternating stages (group grp generates stage grp of every
    // block, warp w K-steps 2h, 2h + 1 with h = (w >> 2) & 1), so that one group's barrier
    // waits overlap the other group's arithmetic; group 0 drains. (For split tiles, whose
    // contraction takes three times as long, the same groups measured 4-8 % slower with three
    // tensor-memory slots.)
    constexpr int NST = GROUPS == 2 ? 1 : 2;  // stages of a block that a warp generates
    constexpr int NKS = GROUPS == 2 ? 2 : 1;  // K-steps of a stage that a warp generates
    constexpr int NDT = GEN_PER_STAGE * 32;   // threads that drain
    const int grp = GROUPS == 2 ? warp >> 3 : 0;
    const int g0 = GROUPS == 2 ? ((warp >> 2) & 1) * 2 : warp >> 2;  // first K-step
    const bool drainer = grp == 0;
    const int row = ((warp & 3) << 5) + lane;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const int cbase = g0 * CW;  // a drainer's coils: [cbase, cbase + NKS CW)
    const uint16_t M1 = 0xBC00u;  // -1 in FP16
    float2* racc = sRacc + threadIdx.x;
    int pending = -1;
    auto flush_pending = [&]() {
      if (pending >= 0) {
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&tfull[pending]));
        pending = -1;
      }
    };
    Ring<NBUF> rb;
    Ring<NSLOT> rs;  // the slot of this warp's next stage
    if (grp == 1) rs.next();
    int seg = 0, seg_pos = 0;  // segments drained; position of the block in its segment
    bool ok = true;
    // the next block's data / the next stage's phases, found ready by a test made during the
    // current stage's arithmetic (so that the test's latency is hidden behind it)
    bool next_full = false, next_pfull = false;
    if (drainer) {
#pragma unroll
      for (int c = 0; c < NKS * CW; ++c) racc[c * NDT] = make_float2(0.f, 0.f);
    }
    bool drain_due = false, d_out = false;
    int d_b = 0, d_slot = 0;
    long long d_row = 0;
    // Add the segment accumulators to the running sums (the E^H pass generated e^{+i phi}:
    // its conjugate is taken here); at the end of a run also write the run's output: per row
    // and coil for both passes.
    auto drain = [&]() -> bool {
      drain_due = false;
      if (!warp_wait(smem_u32(afull), (uint32_t)seg & 1u, abort_flag, p.err, 7, LIM)) return false;
      tc_fence_after();
      const uint32_t lb = tmem + lane_base;
#pragma unroll
      for (int gi = 0; gi < NKS; ++gi) {
        const int cb = cbase + gi * CW;
        float d1r[CW], d1i[CW], d2r[CW], d2i[CW];
        tmem_ld<CW>(lb + cb, d1r);               // D1[:, c]      = A_re B_re
        tmem_ld<CW>(lb + CP + cb, d1i);          // D1[:, C+c]    = A_re B_im
        tmem_ld<CW>(lb + NM + cb, d2r);          // D2[:, c]      = A_im B_re
        tmem_ld<CW>(lb + NM + CP + cb, d2i);     // D2[:, C+c]    = A_im B_im
        if (gi == NKS - 1) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(aempty));
        }
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          float2 a = racc[(gi * CW + c) * NDT];
          if (MODE == ENC) {
            a.x += d1r[c] - d2i[c];
            a.y += d1i[c] + d2r[c];
          } else {
            a.x += d1r[c] + d2i[c];
            a.y += d1i[c] - d2r[c];
          }
          racc[(gi * CW + c) * NDT] = a;
        }
      }
      ++seg;
      if (!d_out) return true;
      // ---------------------------------------------------------------- run output
      // this warp's coils of the run's rows, unscaled (the E^H pass's coil combine with S,
      // Eq. 5, is done when the partial slots are summed)
      const InstDesc& d = desc(d_b);
      float2* dst = d.out + ((long long)d_slot * d.rows_total + d_row) * CP + cbase;
#pragma unroll
      for (int c = 0; c < NKS * CW; ++c) {
        const float sc = d.bscale[cbase + c];
        const float2 a = racc[c * NDT];
        dst[c] = make_float2(a.x * sc, a.y * sc);
      }
#pragma unroll
      for (int c = 0; c < NKS * CW; ++c) racc[c * NDT] = make_float2(0.f, 0.f);
      return true;
    };
    for (;; rb.next()) {
      const int buf = rb.idx;
      if (!next_full && !warp_wait(smem_u32(&full[buf]), rb.phase, abort_flag, p.err, 5, LIM)) {
        ok = false;
        break;
      }
      next_full = false;
      const Meta m = sMeta[buf];
      if (m.flags & META_END) break;
      if (m.flags & META_FIRST) seg_pos = 0;
      const bool seg_last = (m.flags & META_LAST) || seg_pos + 1 == F;
      seg_pos = seg_last ? 0 : seg_pos + 1;
      const InstDesc& dm = desc(m.inst);
      const float2 us2 = make_float2(dm.ph_unscale, dm.ph_unscale);
      const float* anc = sAnc + buf * 128;
      const float ranc = sRowAnc[buf * 128 + row];
      const float2 rb2 = make_float2(ranc, ranc);
      uint4* emit = EMIT ? p.emit + ((long long)m.o * dm.n_inner + m.in) * (16 * 4 * 128) + row
                         : nullptr;
      // stored tiles of this pair: 16 chunks (stage, K-step, half) of [4][128] uint4
      const uint4* ptile =
          STORED ? dm.stored + ((long long)m.o * dm.n_inner + m.in) * (16 * 4 * 128) + row
                 : nullptr;
      for (int sti = 0; sti < NST; ++sti, rs.next()) {
        const int st = GROUPS == 2 ? grp : sti;
        const int slot = rs.idx;
        if (!next_pfull && !warp_wait(smem_u32(&pfull[slot]), rs.phase, abort_flag, p.err, 6, LIM)) {
          ok = false;
          break;
        }
        next_pfull = false;
        tc_fence_after();
#pragma unroll
        for (int gi = 0; gi < NKS; ++gi) {
          const int g = g0 + gi;
          const uint32_t acol = tmem + lane_base + LY::ACOL0 + slot * LY::SLOT_COLS + g * 8;
          if (STORED) {
            // both halves' tiles, loaded before any of them is stored
            uint4 v[2][4];
#pragma unroll
            for (int jh = 0; jh < 2; ++jh) {
              const uint4* c = ptile + (((st * 4 + g) * 2 + jh) * 4) * 128;
              v[jh][0] = __ldg(c);
              v[jh][2] = __ldg(c + 2 * 128);
              if (NPART == 2) {
                v[jh][1] = __ldg(c + 128);
                v[jh][3] = __ldg(c + 3 * 128);
              }
            }
#pragma unroll
            for (int jh = 0; jh < 2; ++jh) {
              const uint32_t re_hi[4] = {v[jh][0].x, v[jh][0].y, v[jh][0].z, v[jh][0].w};
              const uint32_t im_hi[4] = {v[jh][2].x, v[jh][2].y, v[jh][2].z, v[jh][2].w};
              const uint32_t hcol = acol + 4 * jh;
              if (NPART == 2) {
                const uint32_t re_lo[4] = {v[jh][1].x, v[jh][1].y, v[jh][1].z, v[jh][1].w};
                const uint32_t im_lo[4] = {v[jh][3].x, v[jh][3].y, v[jh][3].z, v[jh][3].w};
                tmem_st4(hcol + 0, re_hi);
                tmem_st4(hcol + 32, re_lo);
                tmem_st4(hcol + 64, im_hi);
                tmem_st4(hcol + 96, im_lo);
              } else {
                tmem_st4(hcol + 0, re_hi);
                tmem_st4(hcol + 32, im_hi);
              }
            }
            continue;
          }
          // this thread's 16 phases of K-step g: elements 0..7 in columns [8g, 8g+8), 8..15
          // in [32+8g, ..)
          float dv[16];
          tmem_ld8x2(acol, acol + 32, dv);
#pragma unroll
          for (int jh = 0; jh < 2; ++jh) {
            if (gi == NKS - 1 && jh == 1) {
              // what this warp's next stage waits for: at a block's end the next block's
              // data, and its phases (each barrier observed directly, for the ordering of
              // what it guards)
              const bool block_end = sti == NST - 1;
              if (block_end) {
                const Ring<NBUF> nb = rb.peek();
                next_full = warp_test(smem_u32(&full[nb.idx]), nb.phase);
              }
              const Ring<NSLOT> nr = GROUPS == 2 ? rs.peek().peek() : rs.peek();
              next_pfull =
                  (!block_end || next_full) && warp_test(smem_u32(&pfull[nr.idx]), nr.phase);
            }
            uint32_t re_hi[4], re_lo[4], im_hi[4], im_lo[4];
            const int v0 = st * 64 + g * 16 + 8 * jh;
            const float4 a4 = *reinterpret_cast<const float4*>(anc + v0);
            const float4 a8 = *reinterpret_cast<const float4*>(anc + v0 + 4);
            const float2 an[4] = {make_float2(a4.x, a4.y), make_float2(a4.z, a4.w),
                                  make_float2(a8.x, a8.y), make_float2(a8.z, a8.w)};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              // phase (radians) = D + A + B; not range-reduced: |A|, |B| <= pi and |D| is a
              // few turns, within the argument range the sine unit handles at this accuracy
              float2 t = __ffma2_rn(make_float2(dv[8 * jh + 2 * k], dv[8 * jh + 2 * k + 1]),
                                    us2, an[k]);
              t = __fadd2_rn(t, rb2);
              float2 cs, sn;
              __sincosf(t.x, &sn.x, &cs.x);
              __sincosf(t.y, &sn.y, &cs.y);
              re_hi[k] = pack_h2(cs.x, cs.y);
              im_hi[k] = pack_h2(sn.x, sn.y);
              if (NPART == 2) {
                // lo = v - hi exactly in FP32 (hi holds 11 significant bits of v), then FP16
                const uint32_t hc = re_hi[k], hs = im_hi[k];
                re_lo[k] = pack_h2(fma_f16_f32((uint16_t)(hc & 0xFFFFu), M1, cs.x),
                                   fma_f16_f32((uint16_t)(hc >> 16), M1, cs.y));
                im_lo[k] = pack_h2(fma_f16_f32((uint16_t)(hs & 0xFFFFu), M1, sn.x),
                                   fma_f16_f32((uint16_t)(hs >> 16), M1, sn.y));
              }
            }
            __syncwarp();
            const uint32_t hcol = acol + 4 * jh;
            if (NPART == 2) {
              tmem_st4(hcol + 0, re_hi);
              tmem_st4(hcol + 32, re_lo);
              tmem_st4(hcol + 64, im_hi);
              tmem_st4(hcol + 96, im_lo);
              if (EMIT) {
                uint4* dst = emit + (((st * 4 + g) * 2 + jh) * 4) * 128;
                dst[0] = make_uint4(re_hi[0], re_hi[1], re_hi[2], re_hi[3]);
                dst[128] = make_uint4(re_lo[0], re_lo[1], re_lo[2], re_lo[3]);
                dst[256] = make_uint4(im_hi[0], im_hi[1], im_hi[2], im_hi[3]);
                dst[384] = make_uint4(im_lo[0], im_lo[1], im_lo[2], im_lo[3]);
              }
            } else {
              tmem_st4(hcol + 0, re_hi);
              tmem_st4(hcol + 32, im_hi);
            }
          }
        }
        pending = slot;
        flush_pending();
        if (sti == 0 && drain_due && !drain()) {
          ok = false;
          break;
        }
      }
      if (!ok) break;
      if (GROUPS == 2) rs.next();  // past the other group's stage of the block
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty[buf]));
      if (seg_last && drainer) {
        // drain after this warp's next stage has been generated (or at the end)
        drain_due = true;
        d_out = (m.flags & META_LAST) != 0;
        d_b = m.inst;
        d_slot = m.slot;
        d_row = (long long)m.o * 128 + row;
      }
    }
    if (ok && drain_due) {
      flush_pending();
      ok = drain();
    }
    if (ok) flush_pending();
    // after a time-out, stores of the stage in progress may still be in flight
    tmem_st_wait();
    (void)ok;
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == MMA_WARP) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

template <int MODE, int CP, int NPART, int NKP, bool EMIT>
static int set_smem() {
  static bool attr_set = false;  // per instantiation
  if (!attr_set) {
    SENSE_CUDA_TRY(cudaFuncSetAttribute(tcp_pass_kernel<MODE, CP, NPART, NKP, EMIT>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem_bytes<CP, NPART, NKP>()));
    attr_set = true;
  }
  return SENSE_OK;
}

template <int MODE, int CP, int NPART, int NKP>
static int launch(sense_plan_s* P, const Params& prm, int G, cudaStream_t st) {
  constexpr size_t smem = smem_bytes<CP, NPART, NKP>();
  static_assert(smem <= 232448, "shared memory of the tensor-core phase kernel");
  // tiles are emitted only by a generating split pass (the stored-P set-up)
  constexpr bool CAN_EMIT = NPART == 2 && NKP > 0;
  const bool emit = CAN_EMIT && prm.emit != nullptr;
  if (!CAN_EMIT && prm.emit != nullptr)
    return set_error(SENSE_EUNSUPPORTED, "tile emission needs a generating split pass");
  auto kern = emit ? tcp_pass_kernel<MODE, CP, NPART, NKP, CAN_EMIT>
                   : tcp_pass_kernel<MODE, CP, NPART, NKP, false>;
  int rc = emit ? set_smem<MODE, CP, NPART, NKP, CAN_EMIT>()
                : set_smem<MODE, CP, NPART, NKP, false>();
  if (rc != SENSE_OK) return rc;
  rc = prof_begin(P, MODE == ENC ? KC_TC_ENC : KC_TC_ADJ, st);
  if (rc != SENSE_OK) return rc;
  kern<<<G, NTHREADS, smem, st>>>(prm);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return prof_end(P, st);
}

template <int MODE, int CP, int NPART>
static int by_nkp(sense_plan_s* P, int nkp, const Params& prm, int G, cudaStream_t st) {
  return nkp == 0   ? launch<MODE, CP, NPART, 0>(P, prm, G, st)
         : nkp == 1 ? launch<MODE, CP, NPART, 1>(P, prm, G, st)
                    : launch<MODE, CP, NPART, 2>(P, prm, G, st);
}

template <int MODE, int NPART>
static int by_cp(sense_plan_s* P, int cp, int nkp, const Params& prm, int G, cudaStream_t st) {
  switch (cp) {
    case 8: return by_nkp<MODE, 8, NPART>(P, nkp, prm, G, st);
    case 16: return by_nkp<MODE, 16, NPART>(P, nkp, prm, G, st);
    case 32: return by_nkp<MODE, 32, NPART>(P, nkp, prm, G, st);
    default: return set_error(SENSE_EUNSUPPORTED, "tensor-core phase kernel: padded coils > 32");
  }
}

}  // namespace tcp

namespace tc {

bool tcp_covers(int cp, bool stored) {
  (void)stored;  // both the generated and the stored-P passes run here
  return cp <= 32;
}

int tcp_launch(sense_plan_s* P, int mode, int npart, int cp, int nkp, const Params& prm, int G,
               cudaStream_t st) {
  if (nkp < 0 || nkp > 2) return set_error(SENSE_EUNSUPPORTED, "phase K-steps not in {0, 1, 2}");
  if (mode == ENC)
    return npart == 2 ? tcp::by_cp<ENC, 2>(P, cp, nkp, prm, G, st)
                      : tcp::by_cp<ENC, 1>(P, cp, nkp, prm, G, st);
  return npart == 2 ? tcp::by_cp<ADJ, 2>(P, cp, nkp, prm, G, st)
                    : tcp::by_cp<ADJ, 1>(P, cp, nkp, prm, G, st);
}

}  // namespace tc
}  // namespace sense
