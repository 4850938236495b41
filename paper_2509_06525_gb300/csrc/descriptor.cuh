// Radial Chebyshev descriptor C_n(r) of Eq. 2 for one bond, shared by the
// learned-Hamiltonian kernels (mlp.cu) and the environment-network model
// (bands.cu):
//   f_k(r) = (T_k(2 (r/r_cut - 1)^2 - 1) + 1) / 2 * f_c(r),  k = 0..7,
//   C_n(r) = sum_k c^{Z_i Z_j}_{nk} f_k(r),
// with the cosine cutoff f_c and T_k by the three-term recurrence.
#pragma once
#include <cuda_runtime.h>

namespace gputb {

// C_n(r_ij) for one bond (FP32 from the FP64 distance)
__device__ __forceinline__ void bond_descriptor(float r, float rcut, const float *__restrict__ c /*[8][8]*/,
                                                float (&C)[8]) {
  float f[8];
  // (1 + cos(pi r/rc))/2 written as cos^2(pi r/(2 rc)): no cancellation near rc
  const float ch = cospif(0.5f * r / rcut);
  const float fc = r < rcut ? ch * ch : 0.0f;
  const float u = r / rcut - 1.0f;
  const float x = 2.0f * u * u - 1.0f;
  float t0 = 1.0f, t1 = x;
  f[0] = fc;                      // (T_0 + 1)/2 = 1
  f[1] = 0.5f * (t1 + 1.0f) * fc;
#pragma unroll
  for (int k = 2; k < 8; ++k) {
    const float t2 = 2.0f * x * t1 - t0;
    f[k] = 0.5f * (t2 + 1.0f) * fc;
    t0 = t1;
    t1 = t2;
  }
#pragma unroll
  for (int nn = 0; nn < 8; ++nn) {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s = fmaf(c[nn * 8 + k], f[k], s);
    C[nn] = s;
  }
}

__device__ __forceinline__ void load_mixing(float *sc, const float *__restrict__ cmix) {
  for (int k = threadIdx.x; k < 9 * 64; k += blockDim.x) sc[k] = cmix[k];
}

}  // namespace gputb
