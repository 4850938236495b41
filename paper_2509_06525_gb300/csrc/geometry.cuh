// Box geometry shared by the neighbour search and the kernels that
// recompute bond vectors (teacher Hamiltonian, descriptors, MLP features).
//
// The box rows are a1 = (ax,0,0), a2 = (bx,by,0), a3 = (cx,cy,cz).  The
// minimum-image displacement is reduced one lattice direction at a time
// (a3, then a2, then a1).  When every periodic perpendicular width is at
// least 2 r_cut, an image of j closer than r_cut to i, if one exists, is the
// image this reduction returns.  It serves the kernels that recompute bond
// vectors for values (teacher, descriptors, MLP features); neighbour
// membership itself is decided by the search in neighbors.cu.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace gputb {

struct Box {
  double ax, bx, by, cx, cy, cz;
  int p1, p2, p3;  // periodic flags along a1, a2, a3
  double iax, iby, icz;  // reciprocals of ax, by, cz
};

// Validate the box form and the 2 r_cut width rule on the host.
tb_status make_box(const double *box9, const int32_t *pbc, double rcut, Box *out);

__device__ __forceinline__ double3 min_image(const Box &B, double3 d) {
  // the image index only needs to be right, not correctly rounded: multiply
  // by the reciprocal box lengths (the FP64 divide is slow on GB300)
  if (B.p3) {
    const double n3 = rint(d.z * B.icz);
    d.x = __dsub_rn(d.x, __dmul_rn(n3, B.cx));
    d.y = __dsub_rn(d.y, __dmul_rn(n3, B.cy));
    d.z = __dsub_rn(d.z, __dmul_rn(n3, B.cz));
  }
  if (B.p2) {
    const double n2 = rint(d.y * B.iby);
    d.x = __dsub_rn(d.x, __dmul_rn(n2, B.bx));
    d.y = __dsub_rn(d.y, __dmul_rn(n2, B.by));
  }
  if (B.p1) {
    const double n1 = rint(d.x * B.iax);
    d.x = __dsub_rn(d.x, __dmul_rn(n1, B.ax));
  }
  return d;
}

__device__ __forceinline__ double sq_norm(double3 d) {
  return __dadd_rn(__dadd_rn(__dmul_rn(d.x, d.x), __dmul_rn(d.y, d.y)), __dmul_rn(d.z, d.z));
}

// displacement r_j - r_i (minimum image) from AoS positions [N][3]
__device__ __forceinline__ double3 bond_vector(const Box &B, const double *__restrict__ pos, int64_t i,
                                               int64_t j) {
  double3 d;
  d.x = __dsub_rn(__ldg(pos + 3 * j), __ldg(pos + 3 * i));
  d.y = __dsub_rn(__ldg(pos + 3 * j + 1), __ldg(pos + 3 * i + 1));
  d.z = __dsub_rn(__ldg(pos + 3 * j + 2), __ldg(pos + 3 * i + 2));
  return min_image(B, d);
}

// |r_j - r_i|^2 (minimum image) in FP64, equal to sq_norm(bond_vector()) for
// every pair closer than half a periodic width: the image shift is decided
// from FP32 copies of the differences and applied (with the same explicitly
// rounded operations as min_image) only where it is not zero, which saves
// the FP64 multiplies and roundings of the common unshifted case.
__device__ __forceinline__ double bond_r2(const Box &B, const double *__restrict__ pos, int64_t i, int64_t j) {
  double dx = __dsub_rn(__ldg(pos + 3 * j), __ldg(pos + 3 * i));
  double dy = __dsub_rn(__ldg(pos + 3 * j + 1), __ldg(pos + 3 * i + 1));
  double dz = __dsub_rn(__ldg(pos + 3 * j + 2), __ldg(pos + 3 * i + 2));
  if (B.p3) {
    const float n3 = rintf((float)dz * (float)B.icz);
    if (n3 != 0.0f) {
      dx = __dsub_rn(dx, __dmul_rn((double)n3, B.cx));
      dy = __dsub_rn(dy, __dmul_rn((double)n3, B.cy));
      dz = __dsub_rn(dz, __dmul_rn((double)n3, B.cz));
    }
  }
  if (B.p2) {
    const float n2 = rintf((float)dy * (float)B.iby);
    if (n2 != 0.0f) {
      dx = __dsub_rn(dx, __dmul_rn((double)n2, B.bx));
      dy = __dsub_rn(dy, __dmul_rn((double)n2, B.by));
    }
  }
  if (B.p1) {
    const float n1 = rintf((float)dx * (float)B.iax);
    if (n1 != 0.0f) dx = __dsub_rn(dx, __dmul_rn((double)n1, B.ax));
  }
  return sq_norm(make_double3(dx, dy, dz));
}

// r_j - r_i (minimum image) in FP32 for the learned-H features: the
// coordinate differences in FP64 (exact for nearby atoms), the image shift
// decided from their FP32 values and applied in FP64 only when it is not
// zero (a periodic seam), then FP32.  The shift agrees with min_image for
// every pair closer than half a periodic width.
__device__ __forceinline__ float3 bond_vector_f32(const Box &B, const double *__restrict__ pos, int64_t i,
                                                  int64_t j) {
  double dx = __ldg(pos + 3 * j) - __ldg(pos + 3 * i);
  double dy = __ldg(pos + 3 * j + 1) - __ldg(pos + 3 * i + 1);
  double dz = __ldg(pos + 3 * j + 2) - __ldg(pos + 3 * i + 2);
  if (B.p3) {
    const float n3 = rintf((float)dz * (float)B.icz);
    if (n3 != 0.0f) {
      dx -= (double)n3 * B.cx;
      dy -= (double)n3 * B.cy;
      dz -= (double)n3 * B.cz;
    }
  }
  if (B.p2) {
    const float n2 = rintf((float)dy * (float)B.iby);
    if (n2 != 0.0f) {
      dx -= (double)n2 * B.bx;
      dy -= (double)n2 * B.by;
    }
  }
  if (B.p1) {
    const float n1 = rintf((float)dx * (float)B.iax);
    if (n1 != 0.0f) dx -= (double)n1 * B.ax;
  }
  return make_float3((float)dx, (float)dy, (float)dz);
}

// |r|^2 and |r| of an FP32 bond vector (the length of the learned features)
__device__ __forceinline__ float bond_r2_f32(float3 d) { return fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z)); }

__device__ __forceinline__ float bond_length_f32(const Box &B, const double *__restrict__ pos, int64_t i,
                                                 int64_t j) {
  return sqrtf(bond_r2_f32(bond_vector_f32(B, pos, i, j)));
}

}  // namespace gputb
