// Device-side helpers shared by the kernels: reductions and cache-hinted loads.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace cp {

// Streaming load for matrix data read once per SpMV: evict-first, so the
// Krylov vectors (which are re-read every iteration) keep their L2 lines.
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) { return __ldcs(p); }
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
// Read-only gather of x.
template <typename T>
__device__ __forceinline__ T ld_ro(const T* p) {
  return __ldg(p);
}

// Load that bypasses L1 (served by L2, coherent across SMs): for data that
// other blocks of the same kernel wrote (persistent kernels), where L1 lines
// and the read-only path may still hold an older value.
template <typename T>
__device__ __forceinline__ T ld_cg(const T* p) {
  return __ldcg(p);
}
// x gathers: read-only path in ordinary kernels.  Persistent kernels rewrite x
// between phases, so the read-only path is out; they load through L1
// (ld.global.ca), which is coherent enough here: every read of x follows the
// grid barrier's acquire (thread 0's ld.acquire.gpu, then the block barrier),
// and a weak load ordered after an acquire sees every write ordered before the
// matching release (the PTX memory model), whichever SM made it.  L2ONLY keeps
// a persistent kernel's gathers in L2 (ld.global.cg), for a loop where reuse in
// L1 measured no gain.
template <bool COH, bool L2ONLY = false, typename T>
__device__ __forceinline__ T ld_x(const T* p) {
  if constexpr (COH && L2ONLY) return __ldcg(p);
  else if constexpr (COH) return __ldca(p);
  else return __ldg(p);
}

// Eight consecutive entries of an index or value array through the read-only
// path, as 16-byte vector loads (p must be 16-byte aligned).
__device__ __forceinline__ void ld8_ro(const int32_t* p, int32_t (&o)[8]) {
  const int4 a = __ldg(reinterpret_cast<const int4*>(p));
  const int4 b = __ldg(reinterpret_cast<const int4*>(p) + 1);
  o[0] = a.x, o[1] = a.y, o[2] = a.z, o[3] = a.w, o[4] = b.x, o[5] = b.y, o[6] = b.z, o[7] = b.w;
}
__device__ __forceinline__ void ld8_ro(const double* p, double (&o)[8]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p) + k);
    o[2 * k] = a.x, o[2 * k + 1] = a.y;
  }
}
__device__ __forceinline__ void ld8_ro(const float* p, float (&o)[8]) {
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p) + k);
    o[4 * k] = a.x, o[4 * k + 1] = a.y, o[4 * k + 2] = a.z, o[4 * k + 3] = a.w;
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; the result is valid in thread 0.  Every thread must call
// it; smem holds at least blockDim.x / 32 doubles.  Fixed order: deterministic.
__device__ __forceinline__ double block_sum(double v, double* smem) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();  // smem may still be read by a previous call
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    s = lane < nw ? smem[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;
}

// Sum over the block with few FP64 additions, for blocks of a multiple of 128
// threads: the values go to shared memory, 128 threads (one warp per
// scheduler) each add blockDim.x / 128 of them in a fixed order, then a
// shuffle tree and the 4 warp sums.  About 55 warp-wide FP64 adds for 1024
// threads instead of the 165 of a shuffle tree in every warp, which matters
// where the FP64 pipe is the bound.  buf holds blockDim.x + 4 doubles; the
// result is valid in thread 0; every thread must call it.
__device__ __forceinline__ double block_sum_lean(double v, double* buf) {
  const int nt = blockDim.x;
  __syncthreads();  // buf may still be read by a previous call
  buf[threadIdx.x] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 128) {
    s = buf[threadIdx.x];
    for (int k = threadIdx.x + 128; k < nt; k += 128) s += buf[k];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) buf[nt + (threadIdx.x >> 5)] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) s = (buf[nt] + buf[nt + 1]) + (buf[nt + 2] + buf[nt + 3]);
  return s;
}

// block_sum_lean for G values at once: buf holds G * blockDim.x + G doubles;
// v[g] valid in thread 0 on return.  About (12 x 32) FP64 adds per value for a
// 256-thread block instead of a shuffle tree in every warp (about 1,440).
template <int G>
__device__ __forceinline__ void block_sum_multi_lean(double (&v)[G], double* buf) {
  const int nt = blockDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = nt >> 5;
  __syncthreads();  // buf may still be read by a previous call
#pragma unroll
  for (int g = 0; g < G; ++g) buf[g * nt + threadIdx.x] = v[g];
  __syncthreads();
  for (int g = warp; g < G; g += nw) {
    double s = buf[g * nt + lane];
    for (int k = lane + 32; k < nt; k += 32) s += buf[g * nt + k];
    s = warp_sum(s);
    if (lane == 0) buf[G * nt + g] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int g = 0; g < G; ++g) v[g] = buf[G * nt + g];
  }
}

// The same for G values at once (G small): out[g] valid in thread 0.
template <int G>
__device__ __forceinline__ void block_sum_multi(double (&v)[G], double* smem /*G*32*/) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < G; ++g) v[g] = warp_sum(v[g]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int g = 0; g < G; ++g) smem[g * 32 + warp] = v[g];
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      double s = lane < nw ? smem[g * 32 + lane] : 0.0;
      v[g] = warp_sum(s);
    }
  }
}

// Sum of P block partials in fixed order by the whole block; the result is
// returned to every thread.  smem holds at least blockDim.x / 32 + 1 doubles.
__device__ __forceinline__ double reduce_partials(const double* __restrict__ partials, int P,
                                                  double* smem) {
  double s = 0.0;
  for (int i = threadIdx.x; i < P; i += blockDim.x) s += partials[i];
  s = block_sum(s, smem);
  const int last = blockDim.x >> 5;
  if (threadIdx.x == 0) smem[last] = s;
  __syncthreads();
  s = smem[last];
  __syncthreads();
  return s;
}

// Sum of P block partials in fixed order, valid in thread 0 only.  Scalars
// derived from it (alpha, beta) are then formed once by thread 0 and handed to
// the block through shared memory: an FP64 division is a multi-instruction
// sequence on the FP64 pipe, which CG keeps saturated on parts with a reduced
// FP64 rate, so every thread dividing would cost several microseconds a step.
__device__ __forceinline__ double partials_sum0(const double* __restrict__ partials, int P,
                                                double* smem) {
  double s = 0.0;
  for (int i = threadIdx.x; i < P; i += blockDim.x) s += partials[i];
  return block_sum(s, smem);
}

// Sum of P block partials written by other blocks of the same kernel, by one
// warp (lane l adds partials l, l + 32, ... in order, then a fixed shuffle
// tree): every lane holds the same value, and every block gets the same bits.
// Up to 32 * kPartialsPerLane partials (one per SM of a persistent grid), a
// lane issues all of its loads before its first add, so the sum waits for one
// L2 round trip rather than one per load; the order of the adds is the same.
constexpr int kPartialsPerLane = 5;
__device__ __forceinline__ double warp_partials_cg(const double* __restrict__ partials, int P) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  if (P <= 32 * kPartialsPerLane) {
    double v[kPartialsPerLane];
#pragma unroll
    for (int k = 0; k < kPartialsPerLane; ++k)
      v[k] = lane + 32 * k < P ? __ldcg(partials + lane + 32 * k) : 0.0;
#pragma unroll
    for (int k = 0; k < kPartialsPerLane; ++k)
      if (lane + 32 * k < P) s += v[k];
  } else {
    for (int i = lane; i < P; i += 32) s += __ldcg(partials + i);
  }
  return warp_sum(s);
}

template <typename T>
struct Vec2;
template <>
struct Vec2<double> {
  using type = double2;
};
template <>
struct Vec2<float> {
  using type = float2;
};

}  // namespace cp
