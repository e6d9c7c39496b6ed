// Deterministic block reductions shared by the vector kernels: every kernel writes one
// partial per block and the last block to finish sums the partials in block order.
#pragma once
#include <cuda_runtime.h>

namespace sense {

constexpr int VB = 256;  // threads per block of the vector kernels

// ---------------------------------------------------------------------------------------
// Block reduction of N doubles + last-block completion.
// ---------------------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double* sh /* [N][VB/32] */) {
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < N; ++j) sh[j * (VB / 32) + w] = v[j];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double a = 0.0;
      for (int i = 0; i < VB / 32; ++i) a += sh[j * (VB / 32) + i];
      v[j] = a;
    }
}

// Writes this block's sums; returns true (in thread 0 only) if this block finished last, in
// which case tot[] holds the totals over all blocks. The last block adds the partials with all
// its threads (thread t takes partials t, t + VB, ... in order, then the fixed tree of
// block_sum), so the totals depend only on the grid size and are the same on every run.
// Every thread of the block must call it (it synchronises the block).
template <int N>
__device__ __forceinline__ bool finish_sums(double (&v)[N], double* part, unsigned* counter,
                                            double (&tot)[N]) {
  __shared__ bool last;
  __shared__ double sh[N * (VB / 32)];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < N; ++j) part[blockIdx.x * N + j] = v[j];
    __threadfence();
    const unsigned done = atomicAdd(counter, 1u);
    last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double a[N];
#pragma unroll
  for (int j = 0; j < N; ++j) a[j] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] += ((volatile double*)part)[b * N + j];
  block_sum<N>(a, sh);
  if (threadIdx.x != 0) return false;
#pragma unroll
  for (int j = 0; j < N; ++j) tot[j] = a[j];
  *counter = 0u;
  return true;
}

}  // namespace sense
