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

namespace {

// ---------------------------------------------------------------------------
// Positions as FP32 pairs (x = hi + lo to about 2^-48 relative), so that
// kernels form bond vectors and lengths on the FP32 pipes: GB300 issues FP64
// at a small fraction of the FP32 rate.  (Internal linkage: each translation
// unit that launches pos_pair_kernel has its own copy.)
__global__ void pos_pair_kernel(const double *__restrict__ pos, int64_t n, float4 *__restrict__ hi,
                                float4 *__restrict__ lo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  const float hx = (float)x, hy = (float)y, hz = (float)z;
  hi[i] = make_float4(hx, hy, hz, 0.0f);
  lo[i] = make_float4((float)(x - (double)hx), (float)(y - (double)hy), (float)(z - (double)hz), 0.0f);
}

// the box of `Box` with every lattice component as an FP32 pair
struct BoxPair {
  float2 ax, bx, by, cx, cy, cz;
  float iax, iby, icz;
  int p1, p2, p3;
};

inline BoxPair box_pair(const Box &B) {
  auto split = [](double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
  };
  BoxPair P;
  P.ax = split(B.ax);
  P.bx = split(B.bx);
  P.by = split(B.by);
  P.cx = split(B.cx);
  P.cy = split(B.cy);
  P.cz = split(B.cz);
  P.iax = (float)B.iax;
  P.iby = (float)B.iby;
  P.icz = (float)B.icz;
  P.p1 = B.p1;
  P.p2 = B.p2;
  P.p3 = B.p3;
  return P;
}

// a + b as an unevaluated pair (s, e), s + e exact (Knuth's TwoSum)
__device__ __forceinline__ float2 two_sum_f(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return make_float2(s, (a - (s - bb)) + (b - bb));
}

// x = (h, l) minus k (Lh, Ll): the high parts through TwoSum, so that a
// coordinate difference across a periodic seam loses nothing
__device__ __forceinline__ float2 pair_shift(float2 x, float k, float2 L) {
  const float2 t = two_sum_f(x.x, -k * L.x);
  return make_float2(t.x, t.y + (x.y - k * L.y));
}

// r_j - r_i (minimum image, reduced along a3, a2, a1 as bond_vector_f32)
// from FP32-pair positions, each component as an unevaluated pair (h, l)
// that is exact up to the roundings of the low parts; r_i - r_j gives the
// exact negatives (every step is sign-symmetric)
__device__ __forceinline__ void bond_pair_components(const BoxPair &B, const float4 *__restrict__ ph,
                                                     const float4 *__restrict__ pl, int64_t i, int64_t j,
                                                     float2 &dx, float2 &dy, float2 &dz) {
  const float4 hi = __ldg(ph + i), hj = __ldg(ph + j), li = __ldg(pl + i), lj = __ldg(pl + j);
  dx = two_sum_f(hj.x, -hi.x);
  dy = two_sum_f(hj.y, -hi.y);
  dz = two_sum_f(hj.z, -hi.z);
  dx.y += lj.x - li.x;
  dy.y += lj.y - li.y;
  dz.y += lj.z - li.z;
  if (B.p3) {
    const float n3 = rintf((dz.x + dz.y) * B.icz);
    if (n3 != 0.0f) {
      dx = pair_shift(dx, n3, B.cx);
      dy = pair_shift(dy, n3, B.cy);
      dz = pair_shift(dz, n3, B.cz);
    }
  }
  if (B.p2) {
    const float n2 = rintf((dy.x + dy.y) * B.iby);
    if (n2 != 0.0f) {
      dx = pair_shift(dx, n2, B.bx);
      dy = pair_shift(dy, n2, B.by);
    }
  }
  if (B.p1) {
    const float n1 = rintf((dx.x + dx.y) * B.iax);
    if (n1 != 0.0f) dx = pair_shift(dx, n1, B.ax);
  }
  // normalised (|l| at most half an ulp of h): a seam shift leaves the high
  // parts' remainder of about an ulp of the box length in l, whose square
  // would otherwise be missing from r^2
  dx = two_sum_f(dx.x, dx.y);
  dy = two_sum_f(dy.x, dy.y);
  dz = two_sum_f(dz.x, dz.y);
}

// the bond vector rounded to FP32
__device__ __forceinline__ float3 bond_vector_pair(const BoxPair &B, const float4 *__restrict__ ph,
                                                   const float4 *__restrict__ pl, int64_t i, int64_t j) {
  float2 dx, dy, dz;
  bond_pair_components(B, ph, pl, i, j, dx, dy, dz);
  return make_float3(dx.x + dx.y, dy.x + dy.y, dz.x + dz.y);
}

// a^2 of a normalised pair a = (h, l) as a normalised pair (h^2 exactly by
// FMA, 2 h l to FP32 rounding; l^2 is below the result's last bit)
__device__ __forceinline__ float2 pair_square(float2 a) {
  const float p = __fmul_rn(a.x, a.x);
  const float e = fmaf(a.x, a.x, -p) + 2.0f * a.x * a.y;
  const float s = p + e;
  return make_float2(s, e - (s - p));
}

// sum of two pairs (TwoSum of the high parts, the low parts added)
__device__ __forceinline__ float2 pair_add(float2 a, float2 b) {
  const float2 t = two_sum_f(a.x, b.x);
  const float l = t.y + (a.y + b.y);
  const float s = t.x + l;
  return make_float2(s, l - (s - t.x));
}

// |r_j - r_i|^2 as a pair (about 44 significant bits): the same value for
// (i, j) and (j, i)
__device__ __forceinline__ float2 bond_r2_pair(const BoxPair &B, const float4 *__restrict__ ph,
                                               const float4 *__restrict__ pl, int64_t i, int64_t j) {
  float2 dx, dy, dz;
  bond_pair_components(B, ph, pl, i, j, dx, dy, dz);
  return pair_add(pair_add(pair_square(dx), pair_square(dy)), pair_square(dz));
}

}  // namespace

}  // namespace gputb
