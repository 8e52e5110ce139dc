// Deterministic FP64 reductions: warp shuffles, then shared memory, then a
// fixed-order pass over per-CTA partials by the last CTA to finish.
#pragma once
#include <cuda_runtime.h>

namespace amr {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA; the result is valid in every thread.  NT = blockDim.x.
template <int NT>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double wsum[NT / 32];
  __shared__ double total;
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) wsum[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double s = lane < NT / 32 ? wsum[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) total = s;
  }
  __syncthreads();
  return total;
}

// Two sums at once.
template <int NT>
__device__ __forceinline__ void block_sum2(double &a, double &b) {
  __shared__ double wa[NT / 32], wb[NT / 32];
  __shared__ double ta, tb;
  a = warp_sum(a);
  b = warp_sum(b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) { wa[wid] = a; wb[wid] = b; }
  __syncthreads();
  if (wid == 0) {
    double sa = lane < NT / 32 ? wa[lane] : 0.0, sb = lane < NT / 32 ? wb[lane] : 0.0;
    sa = warp_sum(sa);
    sb = warp_sum(sb);
    if (lane == 0) { ta = sa; tb = sb; }
  }
  __syncthreads();
  a = ta;
  b = tb;
}

// After each CTA stored its partial(s): returns true in every thread of the CTA
// that finished last (classic threadfence reduction).  The counter is reset by
// that CTA so the next launch starts from zero.
__device__ __forceinline__ bool last_cta(unsigned int *ticket) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
    if (is_last) *ticket = 0;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// Fixed-order sum of n partials by one CTA (NT threads): each thread sums a
// strided subset in ascending order, then the CTA tree-reduces.
template <int NT>
__device__ __forceinline__ double sum_partials(const volatile double *p, int n) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) s += p[i];
  return block_sum<NT>(s);
}

// Sum of exact products in FP32 pairs (the Dot2 scheme of Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005): the product
// error comes from an FMA, the addition error from TwoSum, and the collected
// errors are carried in a second FP32 word.  The result is accurate as if
// accumulated in twice the working precision; it is converted to FP64 before
// the cross-thread reduction.  For FP64 inputs it is a plain FP64 sum.
struct Acc2 {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    const float s = hi + p;
    const float bb = s - hi;
    const float se = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += se + pe;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <typename T>
struct DotAcc {
  double s = 0.0;
  __device__ __forceinline__ void add_prod(T a, T b) { s += (double)a * (double)b; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
  Acc2 a;
  __device__ __forceinline__ void add_prod(float x, float y) { a.add_prod(x, y); }
  __device__ __forceinline__ double value() const { return a.value(); }
};

}  // namespace amr
