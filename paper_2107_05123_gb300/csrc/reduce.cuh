// Reductions for the Krylov scalars.
//
// FP64 arithmetic has long latency on this part (a block-wide FP64 shared-memory tree costs more
// than the vector update it reduces), so the per-thread and per-warp stages of the dot products
// of FP32 vectors use double-float (float-pair) arithmetic: products are split exactly with an FMA
// (p = a*b, e = fma(a, b, -p)) and sums use Knuth's TwoSum, so a warp's sum carries ~48 bits of
// significand, as an FP64 sum would. Only the 8 warp sums of a block and the block partials are
// added in FP64. FP64 vectors use FP64 throughout (warp shuffles, no shared-memory tree).
//
// Block partials are combined by the last block to finish (atomic ticket) in a fixed order, so
// results do not depend on scheduling.
#pragma once

#include "dfloat.cuh"
#include "internal.h"

namespace chns {

// ---- double-float accumulator (the DF pair of dfloat.cuh; here a faster addition that adds the
// low parts before one renormalisation, enough for sums of same-signed or small terms)

__device__ __forceinline__ DF df_zero() { return DF{0.f, 0.f}; }

// a + b with the rounding error of the high parts kept (TwoSum)
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float bp = s - a.hi;
  const float err = (a.hi - (s - bp)) + (b.hi - bp);
  const float lo = a.lo + b.lo + err;
  const float hi = s + lo;
  return DF{hi, lo - (hi - s)};
}

// acc += a * b with the product split exactly (TwoProduct via FMA)
__device__ __forceinline__ void df_fma(DF& acc, float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  acc = df_add(acc, DF{p, e});
}

__device__ __forceinline__ void df_addf(DF& acc, float a) { acc = df_add(acc, DF{a, 0.f}); }

__device__ __forceinline__ double df_value(DF a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ DF warp_sum(DF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DF w{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
    v = df_add(v, w);
  }
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double acc_value(DF a) { return df_value(a); }
__device__ __forceinline__ double acc_value(double a) { return a; }

// Per-thread accumulators matching the vector type: DF for float, double for double.
template <class T>
struct Acc;
template <>
struct Acc<float> {
  using type = DF;
  __device__ static DF zero() { return df_zero(); }
  __device__ static void fma(DF& a, float x, float y) { df_fma(a, x, y); }
  __device__ static void add(DF& a, float x) { df_addf(a, x); }
};
template <>
struct Acc<DF> {  // element energies of double-float applies, summed in FP64
  using type = double;
  __device__ static double zero() { return 0.0; }
  __device__ static void fma(double& a, DF x, DF y) { a += (double)(x * y); }
  __device__ static void add(double& a, DF x) { a += (double)x; }
};
template <>
struct Acc<double> {
  using type = double;
  __device__ static double zero() { return 0.0; }
  __device__ static void fma(double& a, double x, double y) { a = ::fma(x, y, a); }
  __device__ static void add(double& a, double x) { a += x; }
};

// Block sums of NV accumulators; the totals (double) are valid in thread 0.
template <int NV, int BS, class A>
__device__ __forceinline__ void block_sum(A (&v)[NV], double (&tot)[NV]) {
  __shared__ double ws[NV][BS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const A s = warp_sum(v[k]);
    if (lane == 0) ws[k][warp] = acc_value(s);
  }
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < BS / 32; ++w) t += ws[k][w];
      tot[k] = t;
    }
}

// Sum of the block accumulators over the grid: thread `pub` publishes the block's partials to
// part[k * pstride + blockIdx.x] (the caller keeps `pub` free of other global stores so that its
// fence is cheap), takes a ticket, and the last block adds all partials in a fixed order. No
// thread returns early; returns true in the last block, where out_sh[k] (shared) holds the totals.
template <int NV, int BS, class A>
__device__ __forceinline__ bool block_reduce_ticket(A (&v)[NV], double* __restrict__ part,
                                                    int64_t pstride, unsigned* __restrict__ counter,
                                                    int pub, double (&out_sh)[NV]) {
  __shared__ double tot[NV];
  __shared__ bool last;
  double t0[NV];
  block_sum<NV, BS>(v, t0);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = t0[k];
  __syncthreads();
  if ((int)threadIdx.x == pub) {
#pragma unroll
    for (int k = 0; k < NV; ++k) part[k * pstride + blockIdx.x] = tot[k];
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  const bool is_last = last;
  if (is_last) {
    __threadfence();
    double s[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      s[k] = 0.0;
      for (unsigned b = threadIdx.x; b < gridDim.x; b += BS)
        s[k] += ((volatile double*)part)[k * pstride + b];
    }
    double fin[NV];
    block_sum<NV, BS>(s, fin);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) out_sh[k] = fin[k];
      *counter = 0u;
    }
    __syncthreads();
  }
  return is_last;
}

// Classic form: thread 0 publishes and the last block writes the totals to out[k] (global).
template <int NV, int BS, class A>
__device__ __forceinline__ void block_reduce_finalize(A (&v)[NV], double* __restrict__ part,
                                                      int64_t pstride,
                                                      unsigned* __restrict__ counter,
                                                      double* __restrict__ out) {
  __shared__ double tot[NV];
  if (block_reduce_ticket<NV, BS>(v, part, pstride, counter, 0, tot) && threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = tot[k];
}

}  // namespace chns
