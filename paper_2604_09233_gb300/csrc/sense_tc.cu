// Tensor-core (tcgen05) E and E^H with the encoding matrix generated on the fly (or, in the
// stored-P comparison mode, streamed from HBM).
//
// One kernel template serves both passes. A pass contracts the phase matrix P = e^{i K R}
// (Eq. 4) against a thin complex operand over one of its two dimensions:
//   ENC (s = E m, Eq. 4):    rows = samples, streamed = voxels,  B = Q = S o m
//   ADJ (m = E^H s, Eq. 5):  rows = voxels,  streamed = samples, B = Sigma,
//                            generated tile conjugated, coil sum in the epilogue.
// Per CTA (one per SM, persistent) the warps split into
//   16 generator warps  : compute 128 rows x 64 streamed phases per stage (FP32 phase,
//                         MUFU sin/cos), convert to FP16 (hi, or hi+lo split) and write
//                         them straight into tensor memory as the A operand;
//   1 MMA warp          : issues tcgen05.mma (A from TMEM, B from shared memory) into two
//                         FP32 accumulators D1 = A_re B^T, D2 = A_im B^T;
//   1 loader warp       : bulk-copies (cp.async.bulk) the B tile image, the streamed
//                         block's phase deltas and its anchors into shared memory, and
//                         publishes each stage's (instance, row block, streamed block, run
//                         flags, output slot) in a shared-memory metadata ring.
// B is the real [2C][64] matrix [B_re; B_im] (per-coil power-of-two scaled FP16, prepared
// as a pre-swizzled 128B-K-major image), so D1 and D2 give the complex product:
//   Y_re = D1[:, c] - D2[:, C+c],  Y_im = D1[:, C+c] + D2[:, c].
// The loader's schedule is stream-K for one problem (the (row block, streamed block) pairs
// cut into equal contiguous ranges, one per CTA; a run of pairs with the same row block
// accumulates in TMEM and is written to a partial slot, summed in a fixed order afterwards)
// or, for a batch, an atomic work queue of (instance, row block, chunk) items. In the STORED
// variant the generator warps copy precomputed phase tiles from HBM into tensor memory
// instead of computing them (gen_stored_kernel writes those tiles once).
// Every wait is bounded: on time-out the CTA records an error, drains what it issued,
// frees its tensor memory and returns.
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

#include "sense_ptx.cuh"
#include "sense_tc.cuh"

namespace sense {
namespace tc {

constexpr int NGEN_WARPS = 16;
constexpr int MMA_WARP = 16;
constexpr int LOAD_WARP = 17;
constexpr int NTHREADS = 18 * 32;
constexpr uint32_t TMEM_COLS = 512;

// ---------------------------------------------------------------------------------------
// the pass kernel
// ---------------------------------------------------------------------------------------
template <int CP, int NPART>
struct Smem {
  static constexpr int BROWS = 2 * CP;
  static constexpr int B_HALF_BYTES = NPART * BROWS * 128;  // one 64-wide half
  static constexpr int B_BYTES = 2 * B_HALF_BYTES;           // one streamed block
  // TMEM: accumulators D1, D2 in columns [0, 4 CP); A slots (one 64-wide half block of
  // NPART x {re, im} FP16 matrices, 32 columns each) from ACOL0 to the end of the 512.
  static constexpr uint32_t ACOL0 = 4 * CP > 128 ? 4 * CP : 128;
  static constexpr int NSLOT_FIT = (int)((512 - ACOL0) / (NPART * 64));
  static constexpr int NSLOT = NSLOT_FIT > 4 ? 4 : NSLOT_FIT;
  // shared-memory stages of streamed blocks (three fit below 64 coils)
  static constexpr int NBUFS = CP <= 32 ? 3 : 2;
};

template <int MODE, int CP, int RT, int NPART, bool STORED>
// 18 warps: up to 5 on one SM sub-partition, whose register file holds 16K registers, so
// 96 registers per thread is the ceiling; one CTA per SM. STORED: the generator warps copy
// precomputed phase tiles from HBM into tensor memory instead of computing them (the loader
// then brings only the B image).
__global__ void __launch_bounds__(NTHREADS, 1) tc_pass_kernel(Params p) {
  using SM = Smem<CP, NPART>;
  constexpr int NBUF = SM::NBUFS;
  constexpr int CW = CP / 4;  // coils per warpgroup in the epilogue
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-align the dynamic shared memory base by pointer arithmetic on the __shared__
  // array itself, so the compiler keeps the shared address space (shared-memory loads,
  // not generic ones)
  uint8_t* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* sB = base;                                              // [NBUF][B_BYTES]
  float* sCol = (float*)(sB + NBUF * SM::B_BYTES);                 // [NBUF][RT][128]
  float* sAnc = sCol + NBUF * 128 * RT;                            // [NBUF][128]
  float* sRowAnc = sAnc + NBUF * 128;                              // [NBUF][128]
  float2* sRed = (float2*)(sRowAnc + NBUF * 128);                  // [4][128]
  float2* sRacc = sRed + 4 * 128;                                  // [CP/4][512]
  Meta* sMeta = (Meta*)(sRacc + (CP / 4) * NGEN_WARPS * 32);      // [NBUF]
  uint64_t* bars = (uint64_t*)(sMeta + NBUF);                      // barriers
  uint64_t* full = bars;                      // [NBUF]
  uint64_t* empty = bars + NBUF;              // [NBUF]
  uint64_t* tfull = bars + 2 * NBUF;          // [SM::NSLOT]
  uint64_t* tempty = tfull + SM::NSLOT;       // [SM::NSLOT]
  uint64_t* afull = tempty + SM::NSLOT;       // accumulator full
  uint64_t* aempty = afull + 1;               // accumulator drained
  uint64_t* drain = aempty + 1;               // final MMA drain
  uint64_t* ered = drain + 1;                 // ADJ epilogue: partial sums written
  uint64_t* edone = ered + 1;                 // ADJ epilogue: partial sums consumed
  uint32_t* tmem_slot = (uint32_t*)(edone + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (p.stop && *p.stop != 0.0) return;
  const bool queue = p.inst != nullptr;
  // instance descriptor (kernel parameter space for stream-K, global memory for the queue)
  auto desc = [&](int b) -> const InstDesc& { return queue ? p.inst[b] : p.d0; };

  const long long i = blockIdx.x;
  const int F = p.seg_len;
  const long long LIM = p.wait_limit > 0 ? p.wait_limit : WAIT_LIMIT_CYCLES;

  if (threadIdx.x == 0) {
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(smem_u32(&full[b]), 1);
      mbar_init(smem_u32(&empty[b]), NGEN_WARPS + 1);
    }
    for (int s = 0; s < SM::NSLOT; ++s) {
      mbar_init(smem_u32(&tfull[s]), NGEN_WARPS);
      mbar_init(smem_u32(&tempty[s]), 1);
    }
    mbar_init(smem_u32(afull), 1);
    mbar_init(smem_u32(aempty), NGEN_WARPS);
    mbar_init(smem_u32(drain), 1);
    mbar_init(smem_u32(ered), NGEN_WARPS);
    mbar_init(smem_u32(edone), 4);
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
  const uint32_t D1 = tmem, D2 = tmem + 2 * CP;
  // Tensor memory is not cleared between kernels and may hold non-finite values left by
  // an earlier kernel; an MMA that starts an accumulation must not see them, so the
  // accumulator columns [0, 4 CP) are zeroed before the first MMA (warpgroup g zeroes
  // columns [g CP, (g+1) CP) of its lane quarter).
  if (warp < NGEN_WARPS) {
    const uint32_t zr[4] = {0u, 0u, 0u, 0u};
    const uint32_t base = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (warp >> 2) * CP;
#pragma unroll
    for (int c = 0; c < CP; c += 4) tmem_st4(base + c, zr);
    tmem_st_wait();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  // A run is a maximal range of pairs with the same row block (one output slot); it is
  // cut into segments of at most F pairs. After each segment the FP32 accumulators are
  // read out of TMEM and added to a per-thread running sum; the running sum is written
  // once per run. The loader decides the pairs and passes them on in sMeta.

  if (warp == LOAD_WARP) {
    // ------------------------------------------------------------------ loader
    if (lane == 0) {
      const uint32_t col_bytes = 128u * RT * 4u;
      long long it = 0;   // blocks pushed
      Ring<NBUF> rb;      // ring position of block it
      bool ok = true;
      // claim the next stage buffer and publish its metadata; with data, also issue the
      // stage's bulk copies (the full barrier completes when they land)
      auto push = [&](int b, int o, int in, int flags, int slot) -> bool {
        const int buf = rb.idx;
        if (it >= NBUF &&
            !mbar_wait(smem_u32(&empty[buf]), rb.phase ^ 1u, abort_flag, p.err, 1, LIM))
          return false;
        Meta m;
        m.inst = b; m.o = o; m.in = in; m.flags = flags; m.slot = slot;
        m.pad0 = m.pad1 = m.pad2 = 0;
        sMeta[buf] = m;
        const uint32_t fb = smem_u32(&full[buf]);
        if (flags & META_END) {
          mbar_arrive(fb);
        } else if (p.hold > 0 && i == 0 && it == p.hold - 1) {
          // test of the time-out path: this stage's arrival is never signalled and no copy
          // is issued for it, so every wait on it runs out after LIM cycles
        } else {
          const InstDesc& d = desc(b);
          mbar_arrive_expect_tx(fb, SM::B_BYTES + (STORED ? 0u : col_bytes + 1024u));
          bulk_g2s(smem_u32(sB + buf * SM::B_BYTES), d.Bimg + (long long)in * SM::B_BYTES,
                   SM::B_BYTES, fb);
          if (!STORED) {
            bulk_g2s(smem_u32(sCol + buf * 128 * RT), d.colT + (long long)in * 128 * RT,
                     col_bytes, fb);
            bulk_g2s(smem_u32(sAnc + buf * 128),
                     d.colAnc + (long long)o * d.cols_total + in * 128, 512u, fb);
            bulk_g2s(smem_u32(sRowAnc + buf * 128),
                     d.rowAnc + (long long)in * d.rows_total + (long long)o * 128, 512u, fb);
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
      // wait for the last copies this warp issued (one per buffer) before the CTA can exit
      const long long n = it;
      for (long long k = (n > NBUF ? n - NBUF : 0); k < n; ++k) {
        const int buf = (int)(k % NBUF);
        long long t0 = clock64();
        while (!mbar_try_wait(smem_u32(&full[buf]), (uint32_t)(k / NBUF) & 1u)) {
          if (clock64() - t0 > LIM) {
            atomicCAS(p.err, 0, 9);
            break;
          }
        }
      }
    }
  } else if (warp == MMA_WARP) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(2 * CP);
      Ring<NBUF> rb;
      Ring<SM::NSLOT> rs;
      int seg = 0, seg_pos = 0;  // segments issued; position of the block in its segment
      bool ok = true;
      for (;; rb.next()) {
        const int buf = rb.idx;
        if (!mbar_wait(smem_u32(&full[buf]), rb.phase, abort_flag, p.err, 2, LIM)) {
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
        const uint32_t sbuf = smem_u32(sB + buf * SM::B_BYTES);
        for (int st = 0; st < 2; ++st, rs.next()) {
          const int slot = rs.idx;
          if (!mbar_wait(smem_u32(&tfull[slot]), rs.phase, abort_flag, p.err, 4, LIM)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t acol = tmem + SM::ACOL0 + slot * (NPART * 64);
          const uint32_t bhi = sbuf + st * SM::B_HALF_BYTES;
          const uint32_t blo = bhi + 2 * CP * 128;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t acc = (seg_first && st == 0 && k == 0) ? 0u : 1u;
            const uint64_t dh = desc_sw128(bhi + 32 * k);
            if (NPART == 2) {
              const uint64_t dl = desc_sw128(blo + 32 * k);
              const uint32_t are_hi = acol + 0 + 8 * k, are_lo = acol + 32 + 8 * k;
              const uint32_t aim_hi = acol + 64 + 8 * k, aim_lo = acol + 96 + 8 * k;
              mma_ts(D1, are_hi, dh, idesc, acc);
              mma_ts(D1, are_hi, dl, idesc, 1u);
              mma_ts(D1, are_lo, dh, idesc, 1u);
              mma_ts(D2, aim_hi, dh, idesc, acc);
              mma_ts(D2, aim_hi, dl, idesc, 1u);
              mma_ts(D2, aim_lo, dh, idesc, 1u);
            } else {
              mma_ts(D1, acol + 8 * k, dh, idesc, acc);
              mma_ts(D2, acol + 32 + 8 * k, dh, idesc, acc);
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
      tc_commit(smem_u32(drain));
      long long t0 = clock64();
      while (!mbar_try_wait(smem_u32(drain), 0u)) {
        if (clock64() - t0 > LIM) {
          atomicCAS(p.err, 0, 10);
          break;
        }
      }
    }
  } else {
    // ------------------------------------------------------------------ generators
    // All waits are warp-uniform (lane 0 polls, the outcome is broadcast) so that every
    // .sync.aligned tcgen05 instruction below runs with the whole warp converged.
    const int g = warp >> 2;            // warpgroup: K-step of every 64-wide stage
    const int row = ((warp & 3) << 5) + lane;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const int cbase = g * CW;
    // phase in turns -> radians; the E^H pass generates the conjugate tile
    const float2 ang_scale = MODE == ADJ ? make_float2(-6.283185307179586f, -6.283185307179586f)
                                         : make_float2(6.283185307179586f, 6.283185307179586f);
    const float2 NEG1 = make_float2(-1.f, -1.f);
    float own[RT];
    // per-thread running sum of the run, in shared memory (frees registers for the
    // generator): element c of this thread at racc[c * NGEN_THREADS]
    float2* racc = sRacc + threadIdx.x;
    constexpr int NGT = NGEN_WARPS * 32;
    // TMEM stores of a stage complete while the next stage is computed: the stage's
    // wait::st and "slot full" signal are issued after the first half of the next stage.
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
    Ring<SM::NSLOT> rs;
    int warm = 0;  // stages generated, counted up to NSLOT (a slot's first use has no wait)
    int seg = 0, run = 0, seg_pos = 0;  // segments, runs; position of the block in its segment
    bool ok = true;
    int cur_b = -1, cur_o = -1;
#pragma unroll
    for (int c = 0; c < CW; ++c) racc[c * NGT] = make_float2(0.f, 0.f);
    // A segment's accumulators are drained after the next stage has been generated, so
    // the generators never wait for the tensor core at segment ends.
    bool drain_due = false, d_out = false;
    int d_b = 0, d_slot = 0;
    long long d_row = 0;
    // Add the segment accumulators to the running sums; at the end of a run also write
    // the run's output and clear the running sums.
    auto drain = [&]() -> bool {
      drain_due = false;
      if (!warp_wait(smem_u32(afull), (uint32_t)seg & 1u, abort_flag, p.err, 7, LIM)) return false;
      tc_fence_after();
      float d1r[CW], d1i[CW], d2r[CW], d2i[CW];
      const uint32_t lb = tmem + lane_base;
      tmem_ld<CW>(lb + cbase, d1r);               // D1[:, c]      = A_re B_re
      tmem_ld<CW>(lb + CP + cbase, d1i);          // D1[:, C+c]    = A_re B_im
      tmem_ld<CW>(lb + 2 * CP + cbase, d2r);      // D2[:, c]      = A_im B_re
      tmem_ld<CW>(lb + 3 * CP + cbase, d2i);      // D2[:, C+c]    = A_im B_im
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(aempty));
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        float2 a = racc[c * NGT];
        a.x += d1r[c] - d2i[c];
        a.y += d1i[c] + d2r[c];
        racc[c * NGT] = a;
      }
      ++seg;
      if (!d_out) return true;
      // ---------------------------------------------------------------- run output
      const InstDesc& d = desc(d_b);
      if (MODE == ENC) {
        float2* dst = d.out + ((long long)d_slot * d.rows_total + d_row) * CP + cbase;
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          const float sc = d.bscale[cbase + c];
          const float2 a = racc[c * NGT];
          dst[c] = make_float2(a.x * sc, a.y * sc);
        }
      } else {
        const float2* Srow = d.S + d_row * CP + cbase;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          const float sc = d.bscale[cbase + c];
          const float2 a = racc[c * NGT];
          const float xr = a.x * sc, xi = a.y * sc;
          const float2 sv = Srow[c];
          acc.x = fmaf(sv.x, xr, fmaf(sv.y, xi, acc.x));
          acc.y = fmaf(sv.x, xi, fmaf(-sv.y, xr, acc.y));
        }
        // combine the four warpgroups' coil ranges through shared memory (bounded
        // mbarrier waits, no unbounded named barrier)
        if (run > 0 &&
            !warp_wait(smem_u32(edone), (uint32_t)(run - 1) & 1u, abort_flag, p.err, 8, LIM))
          return false;
        sRed[g * 128 + row] = acc;
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(ered));
        if (g == 0) {
          if (!warp_wait(smem_u32(ered), (uint32_t)run & 1u, abort_flag, p.err, 8, LIM)) return false;
          float2 v = sRed[row];
          for (int k = 1; k < 4; ++k) {
            v.x += sRed[k * 128 + row].x;
            v.y += sRed[k * 128 + row].y;
          }
          d.out[(long long)d_slot * d.rows_total + d_row] = v;
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(edone));
        }
      }
#pragma unroll
      for (int c = 0; c < CW; ++c) racc[c * NGT] = make_float2(0.f, 0.f);
      ++run;
      return true;
    };
    for (;; rb.next()) {
      const int buf = rb.idx;
      if (!warp_wait(smem_u32(&full[buf]), rb.phase, abort_flag, p.err, 5, LIM)) {
        ok = false;
        break;
      }
      const Meta m = sMeta[buf];
      if (m.flags & META_END) break;
      if (m.flags & META_FIRST) seg_pos = 0;
      const bool seg_last = (m.flags & META_LAST) || seg_pos + 1 == F;
      seg_pos = seg_last ? 0 : seg_pos + 1;
      if (!STORED && (m.o != cur_o || m.inst != cur_b)) {
        cur_o = m.o;
        cur_b = m.inst;
        const float* rT = desc(cur_b).rowT;
#pragma unroll
        for (int q = 0; q < RT; ++q) own[q] = rT[((long long)cur_o * RT + q) * 128 + row];
      }
      // stored tiles of this pair: 16 chunks of [4][128] uint4
      const uint4* ptile =
          STORED ? desc(m.inst).stored +
                       ((long long)m.o * desc(m.inst).n_inner + m.in) * (16 * 4 * 128) + row
                 : nullptr;
      const float* col = sCol + buf * 128 * RT;
      const float* anc = sAnc + buf * 128;
      const float rb = sRowAnc[buf * 128 + row];
      const float2 rb2 = make_float2(rb, rb);
      for (int st = 0; st < 2; ++st, rs.next()) {
        const int slot = rs.idx;
        if (warm < SM::NSLOT) {
          ++warm;
        } else if (!warp_wait(smem_u32(&tempty[slot]), rs.phase ^ 1u, abort_flag, p.err, 6,
                              LIM)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int c0 = st * 64 + g * 16;
        const uint32_t acol = tmem + lane_base + SM::ACOL0 + slot * (NPART * 64) + g * 8;
        if (STORED) {
          // both halves' tiles, loaded before any of them is stored: 2 x (4 | 2) x 16 B
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
            __syncwarp();
            if (jh == 0) flush_pending();
            const uint32_t hc = acol + 4 * jh;
            if (NPART == 2) {
              const uint32_t re_lo[4] = {v[jh][1].x, v[jh][1].y, v[jh][1].z, v[jh][1].w};
              const uint32_t im_lo[4] = {v[jh][3].x, v[jh][3].y, v[jh][3].z, v[jh][3].w};
              tmem_st4(hc + 0, re_hi);
              tmem_st4(hc + 32, re_lo);
              tmem_st4(hc + 64, im_hi);
              tmem_st4(hc + 96, im_lo);
            } else {
              tmem_st4(hc + 0, re_hi);
              tmem_st4(hc + 32, im_hi);
            }
          }
        } else
        // two halves of 8 streamed elements (4 TMEM columns per matrix each)
#pragma unroll
        for (int jh = 0; jh < 2; ++jh) {
          uint32_t re_hi[4], re_lo[4], im_hi[4], im_lo[4];
          {
            // 8 streamed elements as 4 independent two-element chains
            const int v0 = c0 + 8 * jh;
            const float4 a4 = *reinterpret_cast<const float4*>(anc + v0);
            const float4 a8 = *reinterpret_cast<const float4*>(anc + v0 + 4);
            // theta (turns) = A + B + sum_q own_q * delta_q, two pairs per instruction
            float2 t[4];
            t[0] = __fadd2_rn(make_float2(a4.x, a4.y), rb2);
            t[1] = __fadd2_rn(make_float2(a4.z, a4.w), rb2);
            t[2] = __fadd2_rn(make_float2(a8.x, a8.y), rb2);
            t[3] = __fadd2_rn(make_float2(a8.z, a8.w), rb2);
#pragma unroll
            for (int q = 0; q < RT; ++q) {
              const float4 dd = *reinterpret_cast<const float4*>(col + q * 128 + v0);
              const float4 e = *reinterpret_cast<const float4*>(col + q * 128 + v0 + 4);
              const float2 o2 = make_float2(own[q], own[q]);
              t[0] = __ffma2_rn(o2, make_float2(dd.x, dd.y), t[0]);
              t[1] = __ffma2_rn(o2, make_float2(dd.z, dd.w), t[1]);
              t[2] = __ffma2_rn(o2, make_float2(e.x, e.y), t[2]);
              t[3] = __ffma2_rn(o2, make_float2(e.z, e.w), t[3]);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              // radians (sign: conjugate tile for the E^H pass). No range reduction: |A|,
              // |B| <= 1/2 turn, so |theta| <= 1 + |D| turns, and the argument error the
              // sine unit adds for it, about |theta| 2^-24 turn, is of the order of the FP32
              // rounding D already carries and of the unit's own error
              const float2 ang = __fmul2_rn(t[k], ang_scale);
              float2 cs, sn;
              __sincosf(ang.x, &sn.x, &cs.x);
              __sincosf(ang.y, &sn.y, &cs.y);
              if (NPART == 2) {
                // hi = value rounded to 11 significant bits on the integer pipe (exact in
                // FP16 for |v| <= 1), lo = value - hi on the FMA pipe
                const float2 hc = hi11(cs), hs = hi11(sn);
                re_hi[k] = pack_h2(hc.x, hc.y);
                im_hi[k] = pack_h2(hs.x, hs.y);
                const float2 lc = __ffma2_rn(hc, NEG1, cs), ls = __ffma2_rn(hs, NEG1, sn);
                re_lo[k] = pack_h2(lc.x, lc.y);
                im_lo[k] = pack_h2(ls.x, ls.y);
              } else {
                re_hi[k] = pack_h2(cs.x, cs.y);
                im_hi[k] = pack_h2(sn.x, sn.y);
              }
            }
          }
          __syncwarp();
          if (jh == 0) flush_pending();
          const uint32_t hc = acol + 4 * jh;
          if (NPART == 2) {
            tmem_st4(hc + 0, re_hi);
            tmem_st4(hc + 32, re_lo);
            tmem_st4(hc + 64, im_hi);
            tmem_st4(hc + 96, im_lo);
          } else {
            tmem_st4(hc + 0, re_hi);
            tmem_st4(hc + 32, im_hi);
          }
        }
        pending = slot;
        if (st == 0 && drain_due && !drain()) {
          ok = false;
          break;
        }
      }
      if (!ok) break;
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty[buf]));
      if (seg_last) {
        // drain after the next stage has been generated (or at the end)
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
    // after a time-out, stores of the stage in progress may still be in flight: complete
    // them before the tensor memory is released
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

template <int CP, int RP, int NPART>
constexpr size_t smem_bytes() {
  constexpr int NB = Smem<CP, NPART>::NBUFS;
  return 1024 + NB * Smem<CP, NPART>::B_BYTES + NB * 128 * RP * 4 + 2 * NB * 128 * 4 +
         4 * 128 * 8 + (CP / 4) * NGEN_WARPS * 32 * 8 + NB * sizeof(Meta) + 24 * 8 + 16;
}

// ---------------------------------------------------------------------------------------
// B-operand images: per-coil power-of-two scaling, FP16 hi (+ lo), 128B-swizzled rows
// ---------------------------------------------------------------------------------------
// colmax[c] = max over the rows of max(|re|, |im|) of v(r, c) (float bits, >= 0): a
// shared-memory maximum per block, then one global atomic per coil and block
__global__ void colmax_kernel(const float2* __restrict__ src, const float2* __restrict__ S,
                              const float2* __restrict__ pv, long long nrows, int CP,
                              unsigned* __restrict__ colmax) {
  __shared__ unsigned sm[64];
  for (int c = threadIdx.x; c < CP; c += blockDim.x) sm[c] = 0u;
  __syncthreads();
  const long long n = nrows * CP;
  // blockDim.x is a multiple of CP, so a thread keeps one coil for its whole stride
  const int c = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) % CP);
  float mx = 0.0f;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    float2 v;
    if (src) {
      v = src[idx];
    } else {
      const float2 s = S[idx], m = pv[idx / CP];
      v = make_float2(s.x * m.x - s.y * m.y, s.x * m.y + s.y * m.x);
    }
    mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  if (mx > 0.0f) atomicMax(&sm[c], __float_as_uint(mx));
  __syncthreads();
  for (int k = threadIdx.x; k < CP; k += blockDim.x)
    if (sm[k]) atomicMax(&colmax[k], sm[k]);
}

// One thread per 16-byte chunk (8 consecutive rows r of one image row n, one part).
template <int NPART>
__global__ void image_kernel(const float2* __restrict__ src, const float2* __restrict__ S,
                             const float2* __restrict__ pv, long long nrows, int CP,
                             const unsigned* __restrict__ colmax, float* __restrict__ bscale,
                             uint8_t* __restrict__ img) {
  const int BROWS = 2 * CP;
  const long long nchunks = (nrows / 8) * BROWS * NPART;
  if (blockIdx.x == 0 && threadIdx.x < CP) {
    const float mx = __uint_as_float(colmax[threadIdx.x]);
    int e = 0;
    if (mx > 0.0f) frexpf(mx, &e);
    bscale[threadIdx.x] = mx > 0.0f ? ldexpf(1.0f, e - 15) : 1.0f;
  }
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nchunks;
       idx += (long long)gridDim.x * blockDim.x) {
    // idx -> (row chunk rc = rows rc*8..rc*8+7, image row n, part)
    const int part = (int)(idx % NPART);
    const int n = (int)((idx / NPART) % BROWS);
    const long long rc = idx / (NPART * BROWS);
    const int c = n % CP;
    const bool im = n >= CP;
    const float mx = __uint_as_float(colmax[c]);
    int e = 0;
    if (mx > 0.0f) frexpf(mx, &e);
    const float scale = mx > 0.0f ? ldexpf(1.0f, 15 - e) : 1.0f;
    uint32_t words[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float vv[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const long long r = rc * 8 + 2 * k + h;
        float2 v;
        if (src) {
          v = src[r * CP + c];
        } else {
          const float2 s = S[r * CP + c], m = pv[r];
          v = make_float2(s.x * m.x - s.y * m.y, s.x * m.y + s.y * m.x);
        }
        const float x = (im ? v.y : v.x) * scale;
        if (part == 0) {
          vv[h] = x;
        } else {
          vv[h] = x - __half2float(__float2half_rn(x));
        }
      }
      words[k] = pack_h2(vv[0], vv[1]);
    }
    // placement: block b = r / 128, half = (r % 128) / 64, element e = r % 64
    const long long r0 = rc * 8;
    const long long b = r0 / 128;
    const int half = (int)((r0 % 128) / 64);
    const int chunk = (int)((r0 % 64) / 8);
    const long long off = (((b * 2 + half) * NPART + part) * BROWS + n) * 128 +
                          (long long)((chunk ^ (n & 7)) * 16);
    *reinterpret_cast<uint4*>(img + off) = make_uint4(words[0], words[1], words[2], words[3]);
  }
}

}  // namespace tc

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
// Stream-K over chunks of `ch` streamed blocks: chunk by chunk, CTA i takes the pairs
// [iW/G, (i+1)W/G) of the chunk's (row block, streamed block) space (W = n_outer x chunk
// width). Per row block: its partial slots summed over the chunks; per (chunk, row block): the
// slot base = the row block's slots in earlier chunks minus its first CTA in this chunk, so
// the slot of CTA i is base + i. Every CTA range of a chunk must be non-empty (W >= G): then
// all CTAs between the first and the last contributor of a row block write their slot, and
// the reduction never reads a slot nobody wrote.
static int stream_k_layout(long long n_outer, long long n_inner, long long ch, int G,
                           std::vector<int>& base, std::vector<int>& nslot, int* max_slots) {
  const long long nch = (n_inner + ch - 1) / ch;
  base.assign((size_t)(nch * n_outer), 0);
  nslot.assign((size_t)n_outer, 0);
  for (long long c = 0; c < nch; ++c) {
    const long long wc = std::min(ch, n_inner - c * ch);
    const long long W = n_outer * wc;
    auto cta_of = [&](long long w) { return (int)(((w + 1) * G + W - 1) / W - 1); };
    for (long long o = 0; o < n_outer; ++o) {
      const int a = cta_of(o * wc), b = cta_of((o + 1) * wc - 1);
      base[(size_t)(c * n_outer + o)] = nslot[(size_t)o] - a;
      nslot[(size_t)o] += b - a + 1;
    }
  }
  int mx = 1;
  for (int v : nslot) mx = std::max(mx, v);
  *max_slots = mx;
  return SENSE_OK;
}

// Streamed blocks per stream-K chunk: all of them unless their streamed-side images (B image
// of both stages, hi and lo, plus the phase operand; an upper bound) exceed TC_L2_CHUNK_BYTES,
// then equal chunks below that size, as long as every chunk still gives each of the G CTAs
// at least one pair.
static long long chunk_for_cp(int Cp, long long n_outer, long long n_inner, int G) {
  const long long per_block = 2LL * 2 * 2 * Cp * 128 + 16384;
  long long nch = (n_inner * per_block + TC_L2_CHUNK_BYTES - 1) / TC_L2_CHUNK_BYTES;
  if (nch <= 1) return n_inner;
  const long long ch = (n_inner + nch - 1) / nch;
  nch = (n_inner + ch - 1) / ch;
  const long long last = n_inner - (nch - 1) * ch;
  if (n_outer * last < G) return n_inner;
  return ch;
}

static long long chunk_for(const sense_plan_s* P, long long n_outer, long long n_inner, int G) {
  return chunk_for_cp(P->Cp, n_outer, n_inner, G);
}

template <int MODE, int CP, int RP, int NPART, bool STORED = false>
static int launch_pass(sense_plan_s* P, const tc::Params& prm, int G, cudaStream_t st) {
  constexpr size_t smem = tc::smem_bytes<CP, RP, NPART>();
  auto kern = tc::tc_pass_kernel<MODE, CP, RP, NPART, STORED>;
  static bool attr_set = false;  // per instantiation
  if (!attr_set) {
    SENSE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    attr_set = true;
  }
  int rc = prof_begin(P, MODE == tc::ENC ? KC_TC_ENC : KC_TC_ADJ, st);
  if (rc != SENSE_OK) return rc;
  kern<<<G, tc::NTHREADS, smem, st>>>(prm);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return prof_end(P, st);
}

template <int MODE, int CP, int NPART>
static int dispatch_rp(sense_plan_s* P, int rt, const tc::Params& prm, int G, cudaStream_t st,
                       bool stored) {
  // the stored-tile kernel computes no phases: one instantiation serves every row count
  if (stored) return launch_pass<MODE, CP, 4, NPART, true>(P, prm, G, st);
  switch (rt) {
    case 4: return launch_pass<MODE, CP, 4, NPART>(P, prm, G, st);
    case 6: return launch_pass<MODE, CP, 6, NPART>(P, prm, G, st);
    case 8: return launch_pass<MODE, CP, 8, NPART>(P, prm, G, st);
    case 10: return launch_pass<MODE, CP, 10, NPART>(P, prm, G, st);
    case 12: return launch_pass<MODE, CP, 12, NPART>(P, prm, G, st);
    case 16: return launch_pass<MODE, CP, 16, NPART>(P, prm, G, st);
    case 20: return launch_pass<MODE, CP, 20, NPART>(P, prm, G, st);
    default: return set_error(SENSE_EUNSUPPORTED, "delta rows not in {4,6,8,10,12,16,20}");
  }
}

template <int MODE, int NPART>
static int dispatch_cp(sense_plan_s* P, int cp, int rt, const tc::Params& prm, int G,
                       cudaStream_t st, bool stored) {
  switch (cp) {
    case 8: return dispatch_rp<MODE, 8, NPART>(P, rt, prm, G, st, stored);
    case 16: return dispatch_rp<MODE, 16, NPART>(P, rt, prm, G, st, stored);
    case 32: return dispatch_rp<MODE, 32, NPART>(P, rt, prm, G, st, stored);
    case 64: return dispatch_rp<MODE, 64, NPART>(P, rt, prm, G, st, stored);
    default: return set_error(SENSE_EUNSUPPORTED, "padded coils not in {8,16,32,64}");
  }
}

int tc_launch(sense_plan_s* P, int mode, int npart, int cp, int rt, const tc::Params& prm, int G,
              cudaStream_t st, bool stored) {
  if (tc::tcp_covers(cp, stored))
    return tc::tcp_launch(P, mode, npart, cp, stored ? 0 : P->nkp, prm, G, st);
  if (mode == tc::ENC)
    return npart == 2 ? dispatch_cp<tc::ENC, 2>(P, cp, rt, prm, G, st, stored)
                      : dispatch_cp<tc::ENC, 1>(P, cp, rt, prm, G, st, stored);
  return npart == 2 ? dispatch_cp<tc::ADJ, 2>(P, cp, rt, prm, G, st, stored)
                    : dispatch_cp<tc::ADJ, 1>(P, cp, rt, prm, G, st, stored);
}

int tc_xpart_coils(const sense_plan_s* P) { return tc::tcp_covers(P->Cp, false) ? P->Cp : 1; }

static void tc_free_layout(sense_plan_s* P) {
  cudaFree(P->tc_first_e); cudaFree(P->tc_nslot_e); cudaFree(P->tc_first_a);
  cudaFree(P->tc_nslot_a); cudaFree(P->Ypart_tc); cudaFree(P->Xpart_tc);
  P->tc_first_e = P->tc_nslot_e = P->tc_first_a = P->tc_nslot_a = nullptr;
  P->Ypart_tc = P->Xpart_tc = nullptr;
}

// Stream-K layout for the current grid: per row block, its first contributing CTA and its
// number of partial slots; partial buffers sized for the largest slot count.
static int tc_layout(sense_plan_s* P) {
  tc_free_layout(P);
  // Never more CTAs than (row block, streamed block) pairs: with every CTA range
  // non-empty, all CTAs between the first and the last contributor of a row block write
  // their partial slot, so the reduction never reads a slot nobody wrote.
  P->tc_grid = (int)std::min<long long>(P->tc_grid, (long long)P->nsb * P->nvb);
  std::vector<int> fe, ne, fa, na;
  auto pick = [&](long long n_outer, long long n_inner) -> long long {
    if (P->tc_inner_chunk > 0) return std::min<long long>(P->tc_inner_chunk, n_inner);
    return chunk_for(P, n_outer, n_inner, P->tc_grid);
  };
  P->tc_chunk_e = (int)pick(P->nsb, P->nvb);
  P->tc_chunk_a = (int)pick(P->nvb, P->nsb);
  // every chunk must give each CTA at least one pair (a forced chunk width may need fewer CTAs)
  auto min_pairs = [](long long n_outer, long long n_inner, long long ch) {
    const long long nch = (n_inner + ch - 1) / ch;
    return n_outer * std::min(ch, n_inner - (nch - 1) * ch);
  };
  P->tc_grid = (int)std::min<long long>(
      P->tc_grid, std::min(min_pairs(P->nsb, P->nvb, P->tc_chunk_e),
                           min_pairs(P->nvb, P->nsb, P->tc_chunk_a)));
  stream_k_layout(P->nsb, P->nvb, P->tc_chunk_e, P->tc_grid, fe, ne, &P->tc_slots_e);
  stream_k_layout(P->nvb, P->nsb, P->tc_chunk_a, P->tc_grid, fa, na, &P->tc_slots_a);
  auto up = [&](int** d, const std::vector<int>& h) -> int {
    if (cudaMalloc((void**)d, h.size() * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return set_error(SENSE_ENOMEM, "tc layout");
    }
    SENSE_CUDA_TRY(cudaMemcpy(*d, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice));
    return SENSE_OK;
  };
  int rc;
  if ((rc = up(&P->tc_first_e, fe)) != SENSE_OK) return rc;
  if ((rc = up(&P->tc_nslot_e, ne)) != SENSE_OK) return rc;
  if ((rc = up(&P->tc_first_a, fa)) != SENSE_OK) return rc;
  if ((rc = up(&P->tc_nslot_a, na)) != SENSE_OK) return rc;
  if (cudaMalloc((void**)&P->Ypart_tc, (size_t)P->tc_slots_e * P->Kp * P->Cp * 8) != cudaSuccess ||
      cudaMalloc((void**)&P->Xpart_tc, (size_t)P->tc_slots_a * P->Lp * tc_xpart_coils(P) * 8) !=
          cudaSuccess) {
    cudaGetLastError();
    return set_error(SENSE_ENOMEM, "tc partial buffers");
  }
  return SENSE_OK;
}

int tc_setup(sense_plan_s* P) {
  P->tc_grid_req = P->num_sms;
  P->tc_grid = P->num_sms;
  int rc;
  if ((rc = tc_layout(P)) != SENSE_OK) return rc;
  const size_t img_q = (size_t)P->nvb * 2 * 2 * (2 * P->Cp) * 128;   // sized for NPART = 2
  const size_t img_y = (size_t)P->nsb * 2 * 2 * (2 * P->Cp) * 128;
  auto al = [&](void** d, size_t bytes) -> int {
    if (cudaMalloc(d, bytes) != cudaSuccess) {
      cudaGetLastError();
      return set_error(SENSE_ENOMEM, "tc workspace");
    }
    return SENSE_OK;
  };
  if ((rc = al((void**)&P->Qimg, img_q)) != SENSE_OK) return rc;
  if ((rc = al((void**)&P->Yimg, img_y)) != SENSE_OK) return rc;
  if ((rc = al((void**)&P->qscale, P->Cp * 4)) != SENSE_OK) return rc;
  if ((rc = al((void**)&P->yscale, P->Cp * 4)) != SENSE_OK) return rc;
  if ((rc = al((void**)&P->colmax, 2 * P->Cp * 4)) != SENSE_OK) return rc;
  if ((rc = al((void**)&P->tc_err, 4)) != SENSE_OK) return rc;
  SENSE_CUDA_TRY(cudaMemset(P->tc_err, 0, 4));
  return SENSE_OK;
}

void tc_free(sense_plan_s* P) {
  tc_free_layout(P);
  cudaFree(P->p_enc);
  cudaFree(P->p_adj);
  P->p_enc = P->p_adj = nullptr;
  cudaFree(P->Qimg); cudaFree(P->Yimg); cudaFree(P->qscale);
  cudaFree(P->yscale); cudaFree(P->colmax); cudaFree(P->tc_err);
}

// Segment length of a pass: the tuned value, else 4 blocks for split tiles (the FP32
// accumulation bias of the tensor cores stays well inside the split bar) and 16 for single
// tiles (whose FP16 rounding dominates; fewer drains, 3 % faster at 256 x 256 with 32 coils).
static int tc_seg_for(const sense_plan_s* P, int npart) {
  return P->tc_seg_len > 0 ? P->tc_seg_len : (npart == 2 ? 4 : 16);
}

int tc_set_tuning(sense_plan_s* P, int seg_len, int grid, int inner_chunk) {
  if (seg_len < 0 || seg_len > 64 || grid < 0 || grid > 64 * P->num_sms || inner_chunk < 0)
    return set_error(SENSE_EINVAL, "seg_len must be 0..64, grid 0..64 x SMs, inner_chunk >= 0");
  const int g = grid == 0 ? P->num_sms : grid;
  P->tc_seg_len = seg_len;
  if (g != P->tc_grid_req || inner_chunk != P->tc_inner_chunk) {
    SENSE_CUDA_TRY(cudaDeviceSynchronize());
    P->tc_grid_req = g;
    P->tc_grid = g;
    P->tc_inner_chunk = inner_chunk;
    return tc_layout(P);
  }
  return SENSE_OK;
}

// Y_int[k][c] = sum over the stream-K slots of sample block k/128 (0 for padding);
// optionally the user-layout copy, and the per-coil maxima for the next image.
__global__ void tc_reduce_y_kernel(const float2* __restrict__ Ypart, const int* __restrict__ nslot,
                                   long long K, long long Kp, int C, int Cp,
                                   float2* __restrict__ Y, float2* __restrict__ su,
                                   unsigned* __restrict__ colmax, const double* __restrict__ stop) {
  if (stop && *stop != 0.0) return;
  __shared__ unsigned sm[64];
  if (colmax) {
    for (int c = threadIdx.x; c < Cp; c += blockDim.x) sm[c] = 0u;
    __syncthreads();
  }
  const long long n = Kp * Cp;
  float mx = 0.0f;   // blockDim.x is a multiple of Cp: one coil per thread
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long k = i / Cp;
    const int c = (int)(i % Cp);
    float2 a = make_float2(0.f, 0.f);
    if (k < K && c < C) {
      const int ns = nslot[k / TILE];
      for (int s = 0; s < ns; ++s) {
        const float2 v = Ypart[(long long)s * n + i];
        a.x += v.x;
        a.y += v.y;
      }
    }
    if (Y) Y[i] = a;
    if (su && k < K && c < C) su[k * C + c] = a;
    mx = fmaxf(mx, fmaxf(fabsf(a.x), fabsf(a.y)));
  }
  if (colmax) {
    if (mx > 0.0f)
      atomicMax(&sm[(int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) % Cp)],
                __float_as_uint(mx));
    __syncthreads();
    for (int k = threadIdx.x; k < Cp; k += blockDim.x)
      if (sm[k]) atomicMax(&colmax[k], sm[k]);
  }
}

// q[l] = sum over the stream-K slots of voxel block l/128
// q[l] = sum over the voxel block's slots and the coils of conj(S(l, c)) X(l, c) (Eq. 5's coil
// combine; S includes j): the phase kernel writes per-coil partial rows. One thread per (voxel,
// coil), so that the partial rows and S are read contiguously; the Cp coil lanes of a voxel
// (Cp in {8, 16, 32} divides the warp) are summed with shuffles in a fixed order.
__global__ void tc_reduce_xc_kernel(const float2* __restrict__ Xpart, const int* __restrict__ nslot,
                                    const float2* __restrict__ S, long long Lp, int Cp,
                                    float2* __restrict__ q, const double* __restrict__ stop) {
  if (stop && *stop != 0.0) return;
  const long long n = Lp * Cp;   // a multiple of 32: Lp is a multiple of 128
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const long long i = t / Cp;
    const int ns = nslot[i / TILE];
    float2 x = make_float2(0.f, 0.f);
    for (int s = 0; s < ns; ++s) {
      const float2 v = Xpart[(long long)s * n + t];
      x.x += v.x;
      x.y += v.y;
    }
    const float2 sv = S[t];
    float ar = fmaf(sv.x, x.x, sv.y * x.y), ai = fmaf(sv.x, x.y, -sv.y * x.x);
    for (int o = Cp >> 1; o > 0; o >>= 1) {
      ar += __shfl_xor_sync(0xffffffffu, ar, o);
      ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if ((t & (Cp - 1)) == 0) q[i] = make_float2(ar, ai);
  }
}

__global__ void tc_reduce_x_kernel(const float2* __restrict__ Xpart, const int* __restrict__ nslot,
                                   long long Lp, float2* __restrict__ q,
                                   const double* __restrict__ stop) {
  if (stop && *stop != 0.0) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Lp;
       i += (long long)gridDim.x * blockDim.x) {
    const int ns = nslot[i / TILE];
    float2 a = make_float2(0.f, 0.f);
    for (int s = 0; s < ns; ++s) {
      const float2 v = Xpart[(long long)s * Lp + i];
      a.x += v.x;
      a.y += v.y;
    }
    q[i] = a;
  }
}

static int vgrid(sense_plan_s* P, long long n) {
  return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8 * P->num_sms));
}

int tc_reduce_y(sense_plan_s* P, const float2* Ypart, const int* nslot, float2* Y_int,
                float2* s_user, unsigned* cm, const double* stop, cudaStream_t st) {
  if (cm) SENSE_CUDA_TRY(cudaMemsetAsync(cm, 0, P->Cp * 4, st));
  tc_reduce_y_kernel<<<vgrid(P, P->Kp * P->Cp), 256, 0, st>>>(Ypart, nslot, P->K, P->Kp, P->C,
                                                              P->Cp, Y_int, s_user, cm, stop);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return SENSE_OK;
}

int tc_reduce_x(sense_plan_s* P, const float2* Xpart, const int* nslot, float2* q,
                const double* stop, cudaStream_t st) {
  if (tc_xpart_coils(P) > 1)
    tc_reduce_xc_kernel<<<vgrid(P, P->Lp * P->Cp), 256, 0, st>>>(Xpart, nslot, P->S, P->Lp, P->Cp,
                                                                   q, stop);
  else
    tc_reduce_x_kernel<<<vgrid(P, P->Lp), 256, 0, st>>>(Xpart, nslot, P->Lp, q, stop);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return SENSE_OK;
}

int tc_make_image(sense_plan_s* P, int npart, const float2* src, const float2* pv,
                  long long nrows, unsigned* colmax, float* bscale, uint8_t* img,
                  bool have_colmax, cudaStream_t st) {
  if (!have_colmax) {
    SENSE_CUDA_TRY(cudaMemsetAsync(colmax, 0, P->Cp * 4, st));
    tc::colmax_kernel<<<vgrid(P, nrows * P->Cp), 256, 0, st>>>(src, P->S, pv, nrows, P->Cp, colmax);
    SENSE_CUDA_TRY(cudaGetLastError());
    count_launch(P);
  }
  const long long nchunks = (nrows / 8) * 2 * P->Cp * npart;
  if (npart == 2)
    tc::image_kernel<2><<<vgrid(P, nchunks), 256, 0, st>>>(src, P->S, pv, nrows, P->Cp, colmax,
                                                           bscale, img);
  else
    tc::image_kernel<1><<<vgrid(P, nchunks), 256, 0, st>>>(src, P->S, pv, nrows, P->Cp, colmax,
                                                           bscale, img);
  SENSE_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  return SENSE_OK;
}

static int run_pass(sense_plan_s* P, int mode, int npart, const uint8_t* img, const float* bscale,
                    float2* out, const double* stop, cudaStream_t st) {
  NvtxRange nvtx(mode == tc::ENC ? "sense tensor-core E pass" : "sense tensor-core E^H pass");
  tc::Params prm = {};
  const bool enc = mode == tc::ENC;
  tc::InstDesc& d = prm.d0;
  d.rowT = enc ? P->dKt : P->dRt;
  d.colT = enc ? P->dRt : P->dKt;
  d.rowAnc = enc ? P->Banc : P->Aanc;
  d.colAnc = enc ? P->Aanc : P->Banc;
  d.Bimg = img;
  d.bscale = bscale;
  d.S = P->S;
  d.out = out;
  d.stop = nullptr;
  d.rows_total = enc ? P->Kp : P->Lp;
  d.cols_total = enc ? P->Lp : P->Kp;
  d.n_outer = enc ? P->nsb : P->nvb;
  d.n_inner = enc ? P->nvb : P->nsb;
  d.chunk = d.n_inner;
  d.stored = enc ? P->p_enc : P->p_adj;
  d.rowPh = enc ? P->phK_row : P->phR_row;
  d.colPh = enc ? P->phR_col : P->phK_col;
  d.rowAncR = enc ? P->BancR : P->AancR;
  d.colAncR = enc ? P->AancR : P->BancR;
  d.ph_unscale = P->ph_unscale;
  prm.inst = nullptr;
  prm.first_cta = enc ? P->tc_first_e : P->tc_first_a;
  prm.chunk_inner = enc ? P->tc_chunk_e : P->tc_chunk_a;
  prm.W = (long long)d.n_outer * d.n_inner;
  prm.err = P->tc_err;
  prm.stop = stop;
  prm.seg_len = tc_seg_for(P, npart);
  prm.wait_limit = P->tc_wait_cycles;
  prm.hold = P->tc_test_hold;
  const int G = P->tc_grid;
  return tc_launch(P, mode, npart, P->Cp, P->RT, prm, G, st, d.stored != nullptr);
}

static int npart_of(int prec) { return prec == SENSE_PREC_TC_SPLIT ? 2 : 1; }

// Ypart_tc <- E p (p in plan order); then Y_int / s_user / colmax_y as requested
int tc_encode(sense_plan_s* P, int prec, const float2* p_plan, float2* Y_int, float2* s_user,
              bool want_colmax, const double* stop, cudaStream_t st) {
  const int np = npart_of(prec);
  int rc;
  if ((rc = tc_make_image(P, np, nullptr, p_plan, P->Lp, P->colmax, P->qscale, P->Qimg, false, st)))
    return rc;
  if ((rc = run_pass(P, tc::ENC, np, P->Qimg, P->qscale, P->Ypart_tc, stop, st))) return rc;
  unsigned* cm = want_colmax ? P->colmax + P->Cp : nullptr;
  return tc_reduce_y(P, P->Ypart_tc, P->tc_nslot_e, Y_int, s_user, cm, stop, st);
}

// q <- E^H Y_int (plan order). colmax_ready: P->colmax + Cp already holds Y's maxima.
int tc_adjoint(sense_plan_s* P, int prec, const float2* Y_int, float2* q, bool colmax_ready,
               const double* stop, cudaStream_t st) {
  const int np = npart_of(prec);
  int rc;
  if ((rc = tc_make_image(P, np, Y_int, nullptr, P->Kp, P->colmax + P->Cp, P->yscale, P->Yimg,
                       colmax_ready, st)))
    return rc;
  if ((rc = run_pass(P, tc::ADJ, np, P->Yimg, P->yscale, P->Xpart_tc, stop, st))) return rc;
  return tc_reduce_x(P, P->Xpart_tc, P->tc_nslot_a, q, stop, st);
}

namespace tc {

// Stored-P mode: the phase tiles of one pass, computed once with exactly the pass kernel's
// per-element arithmetic (anchor sum, the delta FMAs in row order, range reduction, MUFU
// sin/cos, FP16 hi/lo split), so a pass that streams them is bit-identical to one that
// generates them. One CTA of 128 threads (one per row) per (row block, streamed block) pair;
// chunk c = (stage, warpgroup, half) holds the 8 streamed elements the pass kernel's warpgroup
// writes to tensor memory at once, for the 4 matrices re hi, re lo, im hi, im lo.
template <int MODE>
__global__ void __launch_bounds__(128) gen_stored_kernel(InstDesc d, int RT, long long W,
                                                         uint4* __restrict__ out) {
  __shared__ float s_col[MAX_RP * 128];
  __shared__ float s_anc[128];
  const int row = threadIdx.x;
  const float ang_scale = MODE == ADJ ? -6.283185307179586f : 6.283185307179586f;
  for (long long w = blockIdx.x; w < W; w += gridDim.x) {
    const int o = (int)(w / d.n_inner), in = (int)(w % d.n_inner);
    __syncthreads();
    for (int i = threadIdx.x; i < RT * 128; i += blockDim.x)
      s_col[i] = d.colT[(long long)in * 128 * RT + i];
    s_anc[row] = d.colAnc[(long long)o * d.cols_total + (long long)in * 128 + row];
    __syncthreads();
    float own[MAX_RP];
    for (int q = 0; q < RT; ++q) own[q] = d.rowT[((long long)o * RT + q) * 128 + row];
    const float rb = d.rowAnc[(long long)in * d.rows_total + (long long)o * 128 + row];
    for (int c = 0; c < 16; ++c) {
      const int st = c >> 3, g = (c >> 1) & 3, jh = c & 1;
      const int v0 = st * 64 + g * 16 + jh * 8;
      uint32_t wv[4][4];
      for (int k = 0; k < 4; ++k) {
        float cs[2], sn[2];
        for (int e = 0; e < 2; ++e) {
          const int v = v0 + 2 * k + e;
          float t = __fadd_rn(s_anc[v], rb);
          for (int q = 0; q < RT; ++q) t = __fmaf_rn(own[q], s_col[q * 128 + v], t);
          const float ang = __fmul_rn(t, ang_scale);
          __sincosf(ang, &sn[e], &cs[e]);
        }
        const float2 hc = hi11(make_float2(cs[0], cs[1])), hs = hi11(make_float2(sn[0], sn[1]));
        wv[0][k] = pack_h2(hc.x, hc.y);
        wv[1][k] = pack_h2(__fmaf_rn(hc.x, -1.0f, cs[0]), __fmaf_rn(hc.y, -1.0f, cs[1]));
        wv[2][k] = pack_h2(hs.x, hs.y);
        wv[3][k] = pack_h2(__fmaf_rn(hs.x, -1.0f, sn[0]), __fmaf_rn(hs.y, -1.0f, sn[1]));
      }
      uint4* dst = out + ((w * 16 + c) * 4) * 128 + row;
      for (int m = 0; m < 4; ++m) dst[m * 128] = make_uint4(wv[m][0], wv[m][1], wv[m][2], wv[m][3]);
    }
  }
}

}  // namespace tc

int tc_store_p(sense_plan_s* P, bool enable, cudaStream_t st) {
  cudaFree(P->p_enc);
  cudaFree(P->p_adj);
  P->p_enc = P->p_adj = nullptr;
  if (!enable) return SENSE_OK;
  const size_t bytes = (size_t)P->nsb * P->nvb * 16 * 4 * 128 * sizeof(uint4);
  if (cudaMalloc((void**)&P->p_enc, bytes) != cudaSuccess ||
      cudaMalloc((void**)&P->p_adj, bytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(P->p_enc);
    cudaFree(P->p_adj);
    P->p_enc = P->p_adj = nullptr;
    return set_error(SENSE_ENOMEM, "stored phase tiles (" + std::to_string(2 * bytes >> 20) +
                                       " MiB)");
  }
  if (tc::tcp_covers(P->Cp, false)) {
    // the tensor-core phase kernel writes the tiles it generates (split FP16) while running
    // an ordinary pass over zeroed B images; its stored-P variant reads them back, so stored
    // and generated passes compute the same bits
    SENSE_CUDA_TRY(cudaMemsetAsync(P->Qimg, 0, (size_t)P->nvb * 2 * 2 * (2 * P->Cp) * 128, st));
    SENSE_CUDA_TRY(cudaMemsetAsync(P->Yimg, 0, (size_t)P->nsb * 2 * 2 * (2 * P->Cp) * 128, st));
    for (int mode = 0; mode < 2; ++mode) {
      const bool enc = mode == tc::ENC;
      tc::Params prm = {};
      tc::InstDesc& d = prm.d0;
      d.rowPh = enc ? P->phK_row : P->phR_row;
      d.colPh = enc ? P->phR_col : P->phK_col;
      d.rowAncR = enc ? P->BancR : P->AancR;
      d.colAncR = enc ? P->AancR : P->BancR;
      d.ph_unscale = P->ph_unscale;
      d.Bimg = enc ? P->Qimg : P->Yimg;
      d.bscale = enc ? P->qscale : P->yscale;
      d.S = P->S;
      d.out = enc ? P->Ypart_tc : P->Xpart_tc;
      d.rows_total = enc ? P->Kp : P->Lp;
      d.cols_total = enc ? P->Lp : P->Kp;
      d.n_outer = enc ? P->nsb : P->nvb;
      d.n_inner = enc ? P->nvb : P->nsb;
      d.chunk = d.n_inner;
      prm.first_cta = enc ? P->tc_first_e : P->tc_first_a;
      prm.chunk_inner = enc ? P->tc_chunk_e : P->tc_chunk_a;
      prm.W = (long long)d.n_outer * d.n_inner;
      prm.err = P->tc_err;
      prm.seg_len = tc_seg_for(P, 2);
      prm.wait_limit = P->tc_wait_cycles;
      prm.emit = enc ? P->p_enc : P->p_adj;
      int rc;
      if ((rc = tc::tcp_launch(P, mode, 2, P->Cp, P->nkp, prm, P->tc_grid, st)) != SENSE_OK)
        return rc;
    }
    return SENSE_OK;
  }
  for (int mode = 0; mode < 2; ++mode) {
    const bool enc = mode == tc::ENC;
    tc::InstDesc d = {};
    d.rowT = enc ? P->dKt : P->dRt;
    d.colT = enc ? P->dRt : P->dKt;
    d.rowAnc = enc ? P->Banc : P->Aanc;
    d.colAnc = enc ? P->Aanc : P->Banc;
    d.rows_total = enc ? P->Kp : P->Lp;
    d.cols_total = enc ? P->Lp : P->Kp;
    d.n_outer = enc ? P->nsb : P->nvb;
    d.n_inner = enc ? P->nvb : P->nsb;
    const long long W = (long long)d.n_outer * d.n_inner;
    const int grid = (int)std::min<long long>(W, 32LL * P->num_sms);
    if (enc)
      tc::gen_stored_kernel<tc::ENC><<<grid, 128, 0, st>>>(d, P->RT, W, P->p_enc);
    else
      tc::gen_stored_kernel<tc::ADJ><<<grid, 128, 0, st>>>(d, P->RT, W, P->p_adj);
    SENSE_CUDA_TRY(cudaGetLastError());
    count_launch(P);
  }
  return SENSE_OK;
}

int tc_check_error(sense_plan_s* P) {
  int e = 0;
  SENSE_CUDA_TRY(cudaMemcpy(&e, P->tc_err, 4, cudaMemcpyDeviceToHost));
  if (e != 0) {
    cudaMemset(P->tc_err, 0, 4);
    return set_error(SENSE_ETIMEOUT, "tensor-core pass timed out waiting (site " +
                                         std::to_string(e) + ")");
  }
  return SENSE_OK;
}

}  // namespace sense

extern "C" int sense_plan_store_p(sense_plan P, int32_t enable, void* stream) {
  if (!P) return sense::set_error(SENSE_EINVAL, "null plan");
  int dev = -1;
  SENSE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != P->device) return sense::set_error(SENSE_EINVAL, "plan belongs to another device");
  cudaStream_t st = (cudaStream_t)stream;
  SENSE_CUDA_TRY(cudaStreamSynchronize(st));
  const int rc = sense::tc_store_p(P, enable != 0, st);
  if (rc != SENSE_OK) return rc;
  SENSE_CUDA_TRY(cudaStreamSynchronize(st));
  return SENSE_OK;
}

extern "C" int sense_diag_chunk_width(int64_t n_outer, int64_t n_inner, int32_t cp, int32_t g,
                                      int64_t* width) {
  if (!width || n_outer < 1 || n_inner < 1 || cp < 1 || g < 1)
    return sense::set_error(SENSE_EINVAL, "sizes must be positive and width non-null");
  *width = sense::chunk_for_cp(cp, n_outer, n_inner, g);
  return SENSE_OK;
}

extern "C" int sense_diag_stream_k_layout(int64_t n_outer, int64_t n_inner, int64_t chunk,
                                          int32_t g, int32_t* slot_base, int32_t* nslot,
                                          int32_t* max_slots) {
  if (!slot_base || !nslot || !max_slots || n_outer < 1 || n_inner < 1 || chunk < 1 || g < 1)
    return sense::set_error(SENSE_EINVAL, "sizes must be positive and outputs non-null");
  const long long nch = (n_inner + chunk - 1) / chunk;
  const long long narrowest = std::min<long long>(chunk, n_inner - (nch - 1) * chunk);
  if (n_outer * narrowest < g)
    return sense::set_error(SENSE_EINVAL, "a chunk gives some CTA no pair");
  std::vector<int> base, ns;
  int mx = 0;
  sense::stream_k_layout(n_outer, n_inner, chunk, g, base, ns, &mx);
  std::copy(base.begin(), base.end(), slot_base);
  std::copy(ns.begin(), ns.end(), nslot);
  *max_slots = mx;
  return SENSE_OK;
}
