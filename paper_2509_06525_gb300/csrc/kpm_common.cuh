// Device helpers shared by the KPM kernels (single and batched): vector
// loads and stores of CPT complex numbers per thread, the SplitMix64 phase
// deviate, compensated dot accumulation and the CTA reduction of moment
// partials.
#pragma once
#include <cstring>

#include "common.cuh"

namespace gputb {
namespace kpmdev {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double phase_uniform(uint64_t seed, uint64_t r, uint64_t i) {
  const uint64_t z = splitmix64(seed ^ splitmix64((r << 32) + i));
  return static_cast<double>(z >> 11) * 0x1.0p-53;
}

// the same deviate truncated to its top 24 bits, exactly representable in
// FP32 (for FP32 vectors: phase error below 2 pi 2^-24)
__device__ __forceinline__ float phase_uniform24(uint64_t seed, uint64_t r, uint64_t i) {
  const uint64_t z = splitmix64(seed ^ splitmix64((r << 32) + i));
  return static_cast<float>(z >> 40) * 0x1.0p-24f;
}

// (cos, sin) of the random phase 2 pi u in the vector precision: FP64
// sincos for FP64 vectors, FP32 sincospi of the 24-bit deviate for FP32
// vectors (the FP64 pipe of GB300 is narrow)
template <typename real>
__device__ __forceinline__ void phase_cis(uint64_t seed, uint64_t r, uint64_t i, real &co, real &sn) {
  if constexpr (sizeof(real) == 8) {
    double s, c;
    sincos(2.0 * M_PI * phase_uniform(seed, r, i), &s, &c);
    co = c;
    sn = s;
  } else {
    float s, c;
    sincospif(2.0f * phase_uniform24(seed, r, i), &s, &c);
    co = c;
    sn = s;
  }
}

// Each thread moves CPT complex numbers of one row: one 8-byte access
// (FP32, CPT = 1) or CPT*8/16 (FP32) / CPT (FP64) 16-byte accesses.
template <typename real, int CPT> struct Vec { using T = float4; static constexpr int kChunks = CPT / 2; };
template <> struct Vec<float, 1> { using T = float2; static constexpr int kChunks = 1; };
template <int CPT> struct Vec<double, CPT> { using T = double2; static constexpr int kChunks = CPT; };

// read-only cached load (neighbour gathers)
template <typename real, int CPT>
__device__ __forceinline__ void ld_gather(const real *p, real (&o)[2 * CPT]) {
  using V = typename Vec<real, CPT>::T;
#pragma unroll
  for (int k = 0; k < Vec<real, CPT>::kChunks; ++k) {
    V t = __ldg(reinterpret_cast<const V *>(p) + k);
    memcpy(o + k * (sizeof(V) / sizeof(real)), &t, sizeof(V));
  }
}
// streaming load / store (each element touched once per step)
template <typename real, int CPT>
__device__ __forceinline__ void ld_stream(const real *p, real (&o)[2 * CPT]) {
  using V = typename Vec<real, CPT>::T;
#pragma unroll
  for (int k = 0; k < Vec<real, CPT>::kChunks; ++k) {
    V t = __ldcs(reinterpret_cast<const V *>(p) + k);
    memcpy(o + k * (sizeof(V) / sizeof(real)), &t, sizeof(V));
  }
}
template <typename real, int CPT>
__device__ __forceinline__ void st_stream(real *p, const real (&v)[2 * CPT]) {
  using V = typename Vec<real, CPT>::T;
#pragma unroll
  for (int k = 0; k < Vec<real, CPT>::kChunks; ++k) {
    V t;
    memcpy(&t, v + k * (sizeof(V) / sizeof(real)), sizeof(V));
    __stcs(reinterpret_cast<V *>(p) + k, t);
  }
}

// Running sum of Re(conj(a) b) over the rows a thread visits.  FP64 vectors
// accumulate in FP64.  FP32 vectors keep a Kahan-compensated FP32 pair
// (Kahan 1965): its error stays within about 2 eps_32 sum|terms| however many
// terms there are, it costs four FP32 additions instead of FP64 work (the
// FP64 pipe of GB300 is far narrower), and the pairs of all threads are then
// summed in FP64.
template <typename real> struct DotAcc;
template <> struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double ar, double ai, double br, double bi) { s = fma(ar, br, fma(ai, bi, s)); }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct DotAcc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float ar, float ai, float br, float bi) {
    const float y = fmaf(ar, br, ai * bi) - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Sum acc over all rows of the CTA for each of the R vectors and write the
// CTA's R partials.  Lanes that share `part` (lane mod TPR) hold the same
// vector components.
template <int R, int CPT>
__device__ __forceinline__ void cta_partial(double (&acc)[CPT], double *out) {
  constexpr int TPR = R / CPT;
  __shared__ double red[kWarps][R];
#pragma unroll
  for (int off = 16; off >= TPR; off >>= 1)
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < TPR)
#pragma unroll
    for (int c = 0; c < CPT; ++c) red[warp][lane * CPT + c] = acc[c];
  __syncthreads();
  if (threadIdx.x < R) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += red[w][threadIdx.x];
    out[threadIdx.x] = s;
  }
}


}  // namespace kpmdev
}  // namespace gputb
