// Deterministic FP64 block reductions with last-block finalisation: every block writes its
// partial sums to part[k * pstride + blockIdx.x]; the last block to finish (atomic ticket) sums
// the partials in a fixed order, writes out[k] and resets the ticket. The result does not depend
// on block scheduling.
#pragma once

#include "internal.h"

namespace chns {

template <int NV, int BS>
__device__ __forceinline__ void block_reduce_finalize(double v[NV], double* __restrict__ part,
                                                      int64_t pstride,
                                                      unsigned* __restrict__ counter,
                                                      double* __restrict__ out) {
  __shared__ double sh[NV][BS];
  __shared__ bool last;
#pragma unroll
  for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int w = BS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) part[k * pstride + blockIdx.x] = sh[k][0];
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += BS)
      s += ((volatile double*)part)[k * pstride + b];
    sh[k][threadIdx.x] = s;
  }
  __syncthreads();
  for (int w = BS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = sh[k][0];
    *counter = 0u;
  }
}

// Like block_reduce_finalize, but (1) the partial is published by thread `pub`, which the caller
// keeps free of global stores so that its fence only waits for the partial itself, and (2) no
// thread returns early: every thread gets `last` (this block finished last) and, in the last
// block, the totals in out_sh[k] (shared; valid after the call).
template <int NV, int BS>
__device__ __forceinline__ bool block_reduce_ticket(double v[NV], double* __restrict__ part,
                                                    int64_t pstride, unsigned* __restrict__ counter,
                                                    int pub, double (&out_sh)[NV]) {
  __shared__ double sh[NV][BS];
  __shared__ bool last;
#pragma unroll
  for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int w = BS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if ((int)threadIdx.x == pub) {
#pragma unroll
    for (int k = 0; k < NV; ++k) part[k * pstride + blockIdx.x] = sh[k][0];
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  const bool is_last = last;
  if (is_last) {
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (unsigned b = threadIdx.x; b < gridDim.x; b += BS)
        s += ((volatile double*)part)[k * pstride + b];
      sh[k][threadIdx.x] = s;
    }
    __syncthreads();
    for (int w = BS / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) out_sh[k] = sh[k][0];
      *counter = 0u;
    }
    __syncthreads();
  }
  return is_last;
}

// Write this block's NV sums to part[k * pstride + blockIdx.x] (no fence, no ticket): a later
// kernel, after the launch boundary, adds the partials with block_sum_partials.
template <int NV, int BS>
__device__ __forceinline__ void block_write_partials(double v[NV], double* __restrict__ part,
                                                     int64_t pstride) {
  __shared__ double sh[NV][BS];
#pragma unroll
  for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int w = BS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) part[k * pstride + blockIdx.x] = sh[k][0];
}

// Sum np partials part[k * pstride + b] (b < np) in a fixed order; every thread of the block
// receives the totals in out[k]. The summation order depends only on np and BS.
template <int NV, int BS>
__device__ __forceinline__ void block_sum_partials(const double* __restrict__ part, int64_t pstride,
                                                   int np, double out[NV]) {
  __shared__ double sh[NV][BS];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double t = 0.0;
    for (int b = threadIdx.x; b < np; b += BS) t += part[k * pstride + b];
    sh[k][threadIdx.x] = t;
  }
  __syncthreads();
  for (int w = BS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = sh[k][0];
  __syncthreads();
}

}  // namespace chns
