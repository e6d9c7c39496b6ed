// s = E m without any device allocation.
//
// Some callers cannot allocate device memory when they call into this library: hosts that
// reserve all GPU memory at start-up and forbid allocation afterwards (an allocation can
// block and synchronise the device, which a fixed-latency pipeline cannot afford), and
// callers embedded in a framework whose own allocator owns the device memory, where a raw
// cudaMalloc would bypass its accounting. They also cannot create a plan, which allocates.
// This entry point serves them: it takes the problem arrays directly (device pointers),
// writes the caller's output, and keeps its only scratch -- the per-split partial sums of
// the FP32 encode kernel -- in a fixed array owned by the library.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "sense_internal.cuh"

namespace sense {
namespace noalloc {

// Partial sums [nsplit][K][CP] complex64: 16 MiB. The device code is loaded lazily, so the
// array is created on a device by the first call there; from then on that device holds it
// until the process exits. Calls share it; calls that overlap on the GPU race.
constexpr size_t SCRATCH_FLOAT2 = (size_t)1 << 21;
static __device__ __align__(256) float2 g_scratch[SCRATCH_FLOAT2];

constexpr int THREADS = 128;  // one sample per thread
constexpr int SUB = 64;       // voxels staged per round
constexpr int MAX_P1 = 24;

// Direct evaluation of Eq. 4 for one sample per thread over a voxel chunk: phase in FP64,
// reduced mod 2 pi, exponential and coil products in FP32; partial sum to scratch.
template <int CP>
__global__ void __launch_bounds__(THREADS) encode_direct_kernel(
    const double* __restrict__ Km, const double* __restrict__ Rm, const float2* __restrict__ S,
    const float* __restrict__ j, const float2* __restrict__ m, int64_t L, int64_t K, int C,
    int P1, int64_t vox_per_split, float2* __restrict__ part) {
  __shared__ double sR[SUB * MAX_P1];
  __shared__ float2 sQ[SUB * CP];
  const int64_t k = (int64_t)blockIdx.x * THREADS + threadIdx.x;
  const int split = blockIdx.y;
  const bool live = k < K;
  double kr[MAX_P1];
#pragma unroll
  for (int p = 0; p < MAX_P1; ++p) kr[p] = (live && p < P1) ? Km[k * P1 + p] * (0.5 / M_PI) : 0.0;
  float2 acc[CP];
#pragma unroll
  for (int c = 0; c < CP; ++c) acc[c] = make_float2(0.f, 0.f);
  const int64_t l_begin = (int64_t)split * vox_per_split;
  const int64_t l_end = std::min<int64_t>(L, l_begin + vox_per_split);
  for (int64_t l0 = l_begin; l0 < l_end; l0 += SUB) {
    const int nv = (int)std::min<int64_t>(SUB, l_end - l0);
    __syncthreads();
    for (int i = threadIdx.x; i < SUB * MAX_P1; i += THREADS) {
      const int v = i / MAX_P1, p = i % MAX_P1;
      sR[i] = (v < nv && p < P1) ? Rm[(int64_t)p * L + l0 + v] : 0.0;
    }
    for (int i = threadIdx.x; i < SUB * CP; i += THREADS) {
      const int v = i / CP, c = i % CP;
      float2 q = make_float2(0.f, 0.f);
      if (v < nv && c < C) {
        const float2 s = S[(l0 + v) * C + c];
        const float2 mv = m[l0 + v];
        const float w = j ? j[l0 + v] : 1.0f;
        q = make_float2((s.x * mv.x - s.y * mv.y) * w, (s.x * mv.y + s.y * mv.x) * w);
      }
      sQ[i] = q;
    }
    __syncthreads();
    for (int v = 0; v < nv; ++v) {
      double t = 0.0;
#pragma unroll
      for (int p = 0; p < MAX_P1; ++p) t = fma(kr[p], sR[v * MAX_P1 + p], t);
      const float th = (float)(t - rint(t));
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
  if (live) {
    float2* out = part + ((int64_t)split * K + k) * CP;
#pragma unroll
    for (int c = 0; c < CP; ++c) out[c] = acc[c];
  }
}

__global__ void reduce_kernel(const float2* __restrict__ part, int nsplit, int64_t K, int C,
                              int CP, float2* __restrict__ s) {
  const int64_t n = K * C;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / C;
    const int c = (int)(i % C);
    float2 a = make_float2(0.f, 0.f);
    for (int sp = 0; sp < nsplit; ++sp) {
      const float2 v = part[((int64_t)sp * K + k) * CP + c];
      a.x += v.x;
      a.y += v.y;
    }
    s[i] = a;
  }
}

// Device address of the scratch array, looked up once per device (cudaGetSymbolAddress
// with that device current, which also loads this file's device code there) and cached for
// the life of the process (it does not survive cudaDeviceReset); a host-side name of a
// __device__ array is not a device address and must never be passed to a kernel.
constexpr int MAX_DEVICES = 64;
static std::atomic<float2*> g_scratch_ptr[MAX_DEVICES];

static int scratch_for_current_device(float2** out) {
  int dev = 0;
  SENSE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return set_error(SENSE_EUNSUPPORTED, "device ordinal >= 64");
  float2* ptr = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!ptr) {
    void* p = nullptr;
    SENSE_CUDA_TRY(cudaGetSymbolAddress(&p, g_scratch));
    ptr = (float2*)p;
    g_scratch_ptr[dev].store(ptr, std::memory_order_release);
  }
  *out = ptr;
  return SENSE_OK;
}

template <int CP>
static void launch(dim3 grid, cudaStream_t st, const double* Km, const double* Rm,
                   const float2* S, const float* j, const float2* m, int64_t L, int64_t K, int C,
                   int P1, int64_t per, float2* part) {
  encode_direct_kernel<CP><<<grid, THREADS, 0, st>>>(Km, Rm, S, j, m, L, K, C, P1, per, part);
}

}  // namespace noalloc
}  // namespace sense

using namespace sense;

extern "C" int sense_encode_noalloc(int64_t L, int64_t K, int32_t C, int32_t P1,
                                    const double* Kmat, const double* Rmat, const float* S,
                                    const float* j, const float* m, float* s, void* stream) {
  using namespace sense::noalloc;
  if (!Kmat || !Rmat || !S || !m || !s) return set_error(SENSE_EINVAL, "null pointer argument");
  if (L < 1 || K < 1 || C < 1 || P1 < 1) return set_error(SENSE_EINVAL, "L, K, C, P1 must be >= 1");
  if (C > MAX_CP || P1 > MAX_P1)
    return set_error(SENSE_EINVAL, "sense_encode_noalloc supports at most 64 coils and 24 basis rows");
  const int CP = C <= 8 ? 8 : C <= 16 ? 16 : C <= 32 ? 32 : 64;
  if ((size_t)K * CP > SCRATCH_FLOAT2)
    return set_error(SENSE_EINVAL,
                     "sense_encode_noalloc: K x padded coils exceeds its fixed scratch of 2^21 "
                     "complex values (16 MiB)");
  const void* ptrs[] = {Kmat, Rmat, S, m, s};
  for (const void* p : ptrs)
    if (!is_device_pointer(p)) return set_error(SENSE_EINVAL, "arrays must be device pointers");
  if (j && !is_device_pointer(j)) return set_error(SENSE_EINVAL, "j must be a device pointer");
  float2* part = nullptr;
  int rc = scratch_for_current_device(&part);
  if (rc != SENSE_OK) return rc;
  // split the voxels so that the partial sums fit the scratch and the grid fills the GPU
  const int64_t nkb = (K + THREADS - 1) / THREADS;
  int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>((L + SUB - 1) / SUB, 2048 / nkb));
  nsplit = std::min<int64_t>(nsplit, (int64_t)(SCRATCH_FLOAT2 / ((size_t)K * CP)));
  nsplit = std::max<int64_t>(1, nsplit);
  const int64_t per = ((L + nsplit - 1) / nsplit + SUB - 1) / SUB * SUB;
  nsplit = (L + per - 1) / per;
  cudaStream_t st = (cudaStream_t)stream;
  const dim3 grid((unsigned)nkb, (unsigned)nsplit);
  const double* Kd = Kmat;
  const double* Rd = Rmat;
  const float2* Sd = (const float2*)S;
  const float2* md = (const float2*)m;
  switch (CP) {
    case 8: launch<8>(grid, st, Kd, Rd, Sd, j, md, L, K, C, P1, per, part); break;
    case 16: launch<16>(grid, st, Kd, Rd, Sd, j, md, L, K, C, P1, per, part); break;
    case 32: launch<32>(grid, st, Kd, Rd, Sd, j, md, L, K, C, P1, per, part); break;
    default: launch<64>(grid, st, Kd, Rd, Sd, j, md, L, K, C, P1, per, part); break;
  }
  SENSE_CUDA_TRY(cudaGetLastError());
  const int64_t n = K * C;
  reduce_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(
      part, (int)nsplit, K, C, CP, (float2*)s);
  SENSE_CUDA_TRY(cudaGetLastError());
  return SENSE_OK;
}
