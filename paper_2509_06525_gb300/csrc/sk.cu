// Multi-orbital (s, p, d) Slater-Koster Hamiltonian and its KPM moments,
// matrix-free (arXiv 2509.06525 Sec. 3: the SK angular factors P_lambda(r_ij)
// of Eq. 1; the paper's 1e8-atom graphene DOS uses an s, p and d model).
//
// Orbitals per atom (9): s, p_x, p_y, p_z, d_xy, d_yz, d_zx, d_{x2-y2},
// d_{3z2-r2}; orbital index 9 i + a.  A stored 9 x 9 FP32 block per pair
// would take 324 B (390 GB at 1e8 atoms); instead each SELL element keeps
// its compressed Slater-Koster form -- direction cosines (l, m, n) and the
// ten two-centre integrals V_k(r) -- in 13 FP32 planes (52 B per pair), and
// the Chebyshev step rebuilds the block in registers from the closed-form
// Slater-Koster table (Slater & Koster 1954, Table I): the 45 entries
// E_ab (a <= b) once each, E_ba = (-1)^(l_a + l_b) E_ab.
//
// KPM on the 9N-dimensional orbital space with one random vector per call
// (complex FP32, [N][9]), the moment-doubling identities and Kahan FP32 /
// FP64 sums reduced in a fixed order; spectral bounds from the Gershgorin
// row sums of the same blocks.
#include <cmath>

#include "geometry.cuh"
#include "kpm_step.cuh"

namespace gputb {
namespace {

constexpr int kNO = 9;          // orbitals per atom
constexpr int kSkThreads = 128;
constexpr float kR3 = 1.7320508075688772f;

// 13 planes: l, m, n, then V_0..V_9 (ss_s, sp_s, pp_s, pp_p, sd_s, pd_s, pd_p, dd_s, dd_p, dd_d)
// the ten SK bond integrals at r = a_cc, passed by value (kernel parameter space)
struct SkV0 {
  float v[10];
};

__global__ void sk_geometry_kernel(const double *__restrict__ pos, int64_t n, int64_t n_slices, Box B,
                                   const int64_t *__restrict__ sp, const int32_t *__restrict__ col, int64_t total,
                                   const SkV0 v0, double a_cc, double beta, double rcut, float *__restrict__ geom) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_slices * 32) return;
  const int64_t sb = sp[i >> 5];
  const int w = static_cast<int>((sp[(i >> 5) + 1] - sb) >> 5);
  int64_t e = sb + (i & 31);
  for (int s = 0; s < w; ++s, e += 32) {
    float g[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) g[k] = 0.0f;
    if (i < n) {
      const int32_t j = col[e];
      if (j != i) {
        const double3 d = bond_vector(B, pos, i, j);
        const double r = sqrt(sq_norm(d));
        if (r < rcut) {
          const double inv = 1.0 / r;
          g[0] = (float)(d.x * inv);
          g[1] = (float)(d.y * inv);
          g[2] = (float)(d.z * inv);
          const double ch = cospi(0.5 * r / rcut);
          const double radial = exp(-beta * (r / a_cc - 1.0)) * ch * ch;
#pragma unroll
          for (int k = 0; k < 10; ++k) g[3 + k] = (float)((double)v0.v[k] * radial);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 13; ++k) geom[(int64_t)k * total + e] = g[k];
  }
}

// Visit the 45 independent entries of the SK block for direction (l, m, n)
// and integrals V: f(a, b, E_ab) with a <= b.
template <typename F>
__device__ __forceinline__ void sk_entries(float l, float m, float n, const float (&V)[10], F &&f) {
  const float ss = V[0], sps = V[1], pps = V[2], ppp = V[3], sds = V[4], pds = V[5], pdp = V[6], dds = V[7],
              ddp = V[8], ddd = V[9];
  const float l2 = l * l, m2 = m * m, n2 = n * n;
  const float lm = l * m, mn = m * n, nl = n * l, lmn = l * m * n;
  const float lmd = l2 - m2;                      // l^2 - m^2
  const float zz = n2 - 0.5f * (l2 + m2);         // n^2 - (l^2 + m^2)/2
  const float ppd = pps - ppp;
  // s row
  f(0, 0, ss);
  f(0, 1, l * sps);
  f(0, 2, m * sps);
  f(0, 3, n * sps);
  f(0, 4, kR3 * lm * sds);
  f(0, 5, kR3 * mn * sds);
  f(0, 6, kR3 * nl * sds);
  f(0, 7, 0.5f * kR3 * lmd * sds);
  f(0, 8, zz * sds);
  // p-p
  f(1, 1, l2 * pps + (1.0f - l2) * ppp);
  f(2, 2, m2 * pps + (1.0f - m2) * ppp);
  f(3, 3, n2 * pps + (1.0f - n2) * ppp);
  f(1, 2, lm * ppd);
  f(1, 3, nl * ppd);
  f(2, 3, mn * ppd);
  // p-d
  const float t3 = kR3 * lmn * pds - 2.0f * lmn * pdp;
  f(1, 4, kR3 * l2 * m * pds + m * (1.0f - 2.0f * l2) * pdp);
  f(1, 5, t3);
  f(1, 6, kR3 * l2 * n * pds + n * (1.0f - 2.0f * l2) * pdp);
  f(2, 4, kR3 * m2 * l * pds + l * (1.0f - 2.0f * m2) * pdp);
  f(2, 5, kR3 * m2 * n * pds + n * (1.0f - 2.0f * m2) * pdp);
  f(2, 6, t3);
  f(3, 4, t3);
  f(3, 5, kR3 * n2 * m * pds + m * (1.0f - 2.0f * n2) * pdp);
  f(3, 6, kR3 * n2 * l * pds + l * (1.0f - 2.0f * n2) * pdp);
  f(1, 7, 0.5f * kR3 * l * lmd * pds + l * (1.0f - lmd) * pdp);
  f(2, 7, 0.5f * kR3 * m * lmd * pds - m * (1.0f + lmd) * pdp);
  f(3, 7, 0.5f * kR3 * n * lmd * pds - n * lmd * pdp);
  f(1, 8, l * zz * pds - kR3 * l * n2 * pdp);
  f(2, 8, m * zz * pds - kR3 * m * n2 * pdp);
  f(3, 8, n * zz * pds + kR3 * n * (l2 + m2) * pdp);
  // d-d
  f(4, 4, 3.0f * l2 * m2 * dds + (l2 + m2 - 4.0f * l2 * m2) * ddp + (n2 + l2 * m2) * ddd);
  f(5, 5, 3.0f * m2 * n2 * dds + (m2 + n2 - 4.0f * m2 * n2) * ddp + (l2 + m2 * n2) * ddd);
  f(6, 6, 3.0f * n2 * l2 * dds + (n2 + l2 - 4.0f * n2 * l2) * ddp + (m2 + n2 * l2) * ddd);
  f(4, 5, 3.0f * l * m2 * n * dds + nl * (1.0f - 4.0f * m2) * ddp + nl * (m2 - 1.0f) * ddd);
  f(4, 6, 3.0f * l2 * mn * dds + mn * (1.0f - 4.0f * l2) * ddp + mn * (l2 - 1.0f) * ddd);
  f(5, 6, 3.0f * mn * n * l * dds + lm * (1.0f - 4.0f * n2) * ddp + lm * (n2 - 1.0f) * ddd);
  f(4, 7, 1.5f * lm * lmd * dds - 2.0f * lm * lmd * ddp + 0.5f * lm * lmd * ddd);
  f(5, 7, 1.5f * mn * lmd * dds - mn * (1.0f + 2.0f * lmd) * ddp + mn * (1.0f + 0.5f * lmd) * ddd);
  f(6, 7, 1.5f * nl * lmd * dds + nl * (1.0f - 2.0f * lmd) * ddp - nl * (1.0f - 0.5f * lmd) * ddd);
  f(4, 8, kR3 * lm * zz * dds - 2.0f * kR3 * lm * n2 * ddp + 0.5f * kR3 * lm * (1.0f + n2) * ddd);
  f(5, 8, kR3 * mn * zz * dds + kR3 * mn * (l2 + m2 - n2) * ddp - 0.5f * kR3 * mn * (l2 + m2) * ddd);
  f(6, 8, kR3 * nl * zz * dds + kR3 * nl * (l2 + m2 - n2) * ddp - 0.5f * kR3 * nl * (l2 + m2) * ddd);
  f(7, 7, 0.75f * lmd * lmd * dds + (l2 + m2 - lmd * lmd) * ddp + (n2 + 0.25f * lmd * lmd) * ddd);
  f(7, 8, 0.5f * kR3 * lmd * zz * dds - kR3 * n2 * lmd * ddp + 0.25f * kR3 * (1.0f + n2) * lmd * ddd);
  f(8, 8, zz * zz * dds + 3.0f * n2 * (l2 + m2) * ddp + 0.75f * (l2 + m2) * (l2 + m2) * ddd);
}

__device__ __forceinline__ int l_of(int a) { return a == 0 ? 0 : (a < 4 ? 1 : 2); }

// sum over the CTA (fixed order: warp shuffles, then the warps in order) -> *out
__device__ __forceinline__ void sk_block_sum(double v, double *out) {
  __shared__ double red[kSkThreads / 32];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < kSkThreads / 32; ++q) s += red[q];
    *out = s;
  }
  __syncthreads();
}

__device__ __forceinline__ void load_geom(const float *__restrict__ geom, int64_t total, int64_t e, float &l, float &m,
                                          float &n, float (&V)[10]) {
  l = __ldcs(geom + e);
  m = __ldcs(geom + total + e);
  n = __ldcs(geom + 2 * total + e);
#pragma unroll
  for (int k = 0; k < 10; ++k) V[k] = __ldcs(geom + (int64_t)(3 + k) * total + e);
}

// One Chebyshev step on the orbital vectors ([N][9] complex FP32):
//   out = alpha ((H - shift) x) - (FIRST ? 0 : prev),  prev may alias out;
// doubling partials of <x|x> and Re <x|out> per CTA (slots idx and idx + stride).
template <bool FIRST>
__global__ void __launch_bounds__(kSkThreads) sk_step_kernel(int64_t n, const int64_t *__restrict__ sp,
                                                             const int32_t *__restrict__ col,
                                                             const float *__restrict__ geom, int64_t total,
                                                             float3 onsite, const float2 *__restrict__ x,
                                                             const float2 *prev, float2 *out,
                                                             double *__restrict__ partial, int64_t slot_stride,
                                                             float alpha, float shift) {
  DotAcc<float> acc, acc2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float2 y[kNO], xi[kNO];
#pragma unroll
    for (int a = 0; a < kNO; ++a) {
      xi[a] = __ldg(x + i * kNO + a);
      const float e = (a == 0 ? onsite.x : (a < 4 ? onsite.y : onsite.z)) - shift;
      y[a] = make_float2(e * xi[a].x, e * xi[a].y);
    }
    const int64_t sb = __ldg(sp + (i >> 5));
    const int w = static_cast<int>((__ldg(sp + (i >> 5) + 1) - sb) >> 5);
    int64_t e = sb + (i & 31);
    for (int s = 0; s < w; ++s, e += 32) {
      const int32_t j = __ldcs(col + e);
      float l, m, nn, V[10];
      load_geom(geom, total, e, l, m, nn, V);
      float2 xj[kNO];
#pragma unroll
      for (int b = 0; b < kNO; ++b) xj[b] = __ldg(x + (int64_t)j * kNO + b);
      sk_entries(l, m, nn, V, [&](int a, int b, float h) {
        y[a].x = fmaf(h, xj[b].x, y[a].x);
        y[a].y = fmaf(h, xj[b].y, y[a].y);
        if (a != b) {
          const float hb = ((l_of(a) + l_of(b)) & 1) ? -h : h;
          y[b].x = fmaf(hb, xj[a].x, y[b].x);
          y[b].y = fmaf(hb, xj[a].y, y[b].y);
        }
      });
    }
#pragma unroll
    for (int a = 0; a < kNO; ++a) {
      float2 o;
      if (FIRST) {
        o = make_float2(alpha * y[a].x, alpha * y[a].y);
      } else {
        const float2 p = __ldcs(prev + i * kNO + a);
        o = make_float2(fmaf(alpha, y[a].x, -p.x), fmaf(alpha, y[a].y, -p.y));
      }
      __stcs(out + i * kNO + a, o);
      acc.add(xi[a].x, xi[a].y, xi[a].x, xi[a].y);
      acc2.add(xi[a].x, xi[a].y, o.x, o.y);
    }
  }
  sk_block_sum(acc.value(), partial + blockIdx.x);
  sk_block_sum(acc2.value(), partial + slot_stride + blockIdx.x);
}

// orbital vectors v0[9 i + a] = exp(2 pi i u(seed, r0, 9 i + a)); partials of <v0|v0>
__global__ void __launch_bounds__(kSkThreads) sk_phase_kernel(int64_t n, uint64_t seed, int64_t r0,
                                                              float2 *__restrict__ v0, double *__restrict__ partial) {
  double acc = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * kNO; t += (int64_t)gridDim.x * blockDim.x) {
    float sn, co;
    phase_cis<float>(seed, (uint64_t)r0, (uint64_t)t, co, sn);
    const float2 v = make_float2(co, sn);
    v0[t] = v;
    acc += (double)v.x * v.x + (double)v.y * v.y;
  }
  sk_block_sum(acc, partial + blockIdx.x);
}

// Gershgorin: per orbital row, onsite +- sum |H_ab| over the row's blocks
__global__ void __launch_bounds__(kSkThreads) sk_gershgorin_kernel(int64_t n, const int64_t *__restrict__ sp,
                                                                   const int32_t *__restrict__ col,
                                                                   const float *__restrict__ geom, int64_t total,
                                                                   float3 onsite, double *__restrict__ lo_part,
                                                                   double *__restrict__ hi_part) {
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float rs[kNO];
#pragma unroll
    for (int a = 0; a < kNO; ++a) rs[a] = 0.0f;
    const int64_t sb = sp[i >> 5];
    const int w = static_cast<int>((sp[(i >> 5) + 1] - sb) >> 5);
    int64_t e = sb + (i & 31);
    for (int s = 0; s < w; ++s, e += 32) {
      float l, m, nn, V[10];
      load_geom(geom, total, e, l, m, nn, V);
      sk_entries(l, m, nn, V, [&](int a, int b, float h) {
        rs[a] += fabsf(h);
        if (a != b) rs[b] += fabsf(h);
      });
    }
#pragma unroll
    for (int a = 0; a < kNO; ++a) {
      const double d = a == 0 ? onsite.x : (a < 4 ? onsite.y : onsite.z);
      // widen by a relative 1e-6 for the FP32 block values
      const double r = (double)rs[a] * (1.0 + 1e-6);
      lo = fmin(lo, d - r);
      hi = fmax(hi, d + r);
    }
  }
  __shared__ double sl[kSkThreads / 32], sh[kSkThreads / 32];
  for (int off = 16; off > 0; off >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, off));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, off));
  }
  if ((threadIdx.x & 31) == 0) {
    sl[threadIdx.x >> 5] = lo;
    sh[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < kSkThreads / 32; ++q) {
      lo = fmin(lo, sl[q]);
      hi = fmax(hi, sh[q]);
    }
    lo_part[blockIdx.x] = fmin(lo, sl[0]);
    hi_part[blockIdx.x] = fmax(hi, sh[0]);
  }
}

__global__ void minmax_reduce_kernel(const double *__restrict__ lo, const double *__restrict__ hi, int parts,
                                     double *__restrict__ out) {
  double a = INFINITY, b = -INFINITY;
  for (int k = threadIdx.x; k < parts; k += blockDim.x) {
    a = fmin(a, lo[k]);
    b = fmax(b, hi[k]);
  }
  for (int off = 16; off > 0; off >>= 1) {
    a = fmin(a, __shfl_xor_sync(0xffffffffu, a, off));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, off));
  }
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}

int sk_grid(int64_t n) {
  static int per_sm = 0;
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sk_step_kernel<false>, kSkThreads, 0) != cudaSuccess ||
        b <= 0)
      b = 4;
    per_sm = b;
  }
  const int64_t need = (n + kSkThreads - 1) / kSkThreads;
  const int64_t cap = (int64_t)per_sm * sm_count();
  return static_cast<int>(need < cap ? need : cap);
}

}  // namespace
}  // namespace gputb

using namespace gputb;

extern "C" tb_status tb_sk_geometry(const double *positions, int64_t n, const double *box, const int32_t *pbc,
                                    double rcut, const int64_t *slice_ptr, const int32_t *col, int64_t total,
                                    const double *v0, double a_cc, double beta, float *geom, void *stream) {
  TB_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "tb_sk_geometry: bad n");
  TB_REQUIRE(positions && slice_ptr && v0 && geom && (total == 0 || col), "tb_sk_geometry: null pointer argument");
  TB_REQUIRE(rcut > 0.0 && a_cc > 0.0, "tb_sk_geometry: need rcut > 0 and a_cc > 0");
  Box B;
  tb_status s = make_box(box, pbc, rcut, &B);
  if (s != TB_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SkV0 hv;
  for (int k = 0; k < 10; ++k) hv.v[k] = (float)v0[k];
  const int64_t n_slices = (n + 31) / 32;
  sk_geometry_kernel<<<(unsigned)((n_slices * 32 + 255) / 256), 256, 0, st>>>(positions, n, n_slices, B, slice_ptr,
                                                                               col, total, hv, a_cc, beta, rcut, geom);
  TB_CHECK_LAUNCH();
  TB_CUDA(cudaStreamSynchronize(st));
  return TB_OK;
}

extern "C" tb_status tb_sk_bounds(int64_t n, const int64_t *slice_ptr, const int32_t *col, const float *geom,
                                  int64_t total, const double *onsite, double *bounds_out, void *workspace,
                                  size_t workspace_bytes, void *stream) {
  TB_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "tb_sk_bounds: bad n");
  TB_REQUIRE(slice_ptr && geom && onsite && bounds_out && workspace, "tb_sk_bounds: null pointer argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int grid = sk_grid(n);
  Carver cv(workspace, workspace_bytes);
  double *lo = cv.take<double>(grid), *hi = cv.take<double>(grid), *out = cv.take<double>(2);
  if (!cv.ok()) return fail(TB_ERR_WORKSPACE, "tb_sk_bounds: workspace too small");
  const float3 on = make_float3((float)onsite[0], (float)onsite[1], (float)onsite[2]);
  sk_gershgorin_kernel<<<grid, kSkThreads, 0, st>>>(n, slice_ptr, col, geom, total, on, lo, hi);
  TB_CHECK_LAUNCH();
  minmax_reduce_kernel<<<1, 32, 0, st>>>(lo, hi, grid, out);
  TB_CHECK_LAUNCH();
  double h[2];
  TB_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, st));
  TB_CUDA(cudaStreamSynchronize(st));
  if (!std::isfinite(h[0]) || !std::isfinite(h[1]) || !(h[1] > h[0]))
    return fail(TB_ERR_NOT_FINITE, "tb_sk_bounds: degenerate or non-finite bounds");
  const double eps = 0.01;
  bounds_out[0] = h[0];
  bounds_out[1] = h[1];
  bounds_out[2] = (h[1] - h[0]) / (2.0 - eps);
  bounds_out[3] = 0.5 * (h[0] + h[1]);
  return TB_OK;
}

extern "C" size_t sk_kpm_workspace_size(int64_t n, int32_t M) {
  if (n <= 0 || M < 2) return 0;
  Carver cv(nullptr, 0);
  for (int k = 0; k < 3; ++k) cv.take<float2>((size_t)n * kNO);
  cv.take<double>((size_t)(M + 1) * sk_grid(n));
  cv.take<int>(4);
  return cv.used + 256;
}

extern "C" tb_status sk_kpm_moments(int64_t n, const int64_t *slice_ptr, const int32_t *col, const float *geom,
                                    int64_t total, const double *onsite, double a, double b, int32_t M, uint64_t seed,
                                    int64_t first_vector, double *mu_out, void *workspace, size_t workspace_bytes,
                                    void *stream, double *ms_out) {
  TB_REQUIRE(n >= 1 && n < (int64_t(1) << 31) / kNO, "sk_kpm_moments: n=%lld out of range", (long long)n);
  TB_REQUIRE(M >= 2, "sk_kpm_moments: M must be >= 2");
  TB_REQUIRE(a > 0.0 && std::isfinite(a) && std::isfinite(b), "sk_kpm_moments: need finite a > 0, b");
  TB_REQUIRE(first_vector >= 0 && first_vector <= (int64_t(1) << 31), "sk_kpm_moments: first_vector out of range");
  TB_REQUIRE(slice_ptr && geom && onsite && mu_out && workspace, "sk_kpm_moments: null pointer argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int grid = sk_grid(n);
  Carver cv(workspace, workspace_bytes);
  float2 *v0 = cv.take<float2>((size_t)n * kNO), *A = cv.take<float2>((size_t)n * kNO),
         *B = cv.take<float2>((size_t)n * kNO);
  double *partial = cv.take<double>((size_t)(M + 1) * grid);
  int *flags = cv.take<int>(4);
  if (!cv.ok()) return fail(TB_ERR_WORKSPACE, "sk_kpm_moments: workspace too small");
  const float3 on = make_float3((float)onsite[0], (float)onsite[1], (float)onsite[2]);
  const float shift = (float)b, inv_a = (float)(1.0 / a), two_over_a = (float)(2.0 / a);
  const int64_t ps = grid;   // partials per slot (R = 1)
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (ms_out) {
    TB_CUDA(cudaEventCreate(&ev[0]));
    TB_CUDA(cudaEventCreate(&ev[1]));
    TB_CUDA(cudaEventRecord(ev[0], st));
  }
  TB_CUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
  sk_phase_kernel<<<grid, kSkThreads, 0, st>>>(n, seed, first_vector, v0, partial);
  TB_CHECK_LAUNCH();
  // doubling: the step reading v_k adds the partials of S_2k and S_2k+1
  sk_step_kernel<true><<<grid, kSkThreads, 0, st>>>(n, slice_ptr, col, geom, total, on, v0, nullptr, A, partial, ps,
                                                    inv_a, shift);
  TB_CHECK_LAUNCH();
  const int last = (M - 1) / 2 + 1;
  for (int m = 2; m <= last; ++m) {
    float2 *out = (m & 1) ? A : B;
    const float2 *x = (m & 1) ? B : A;
    const float2 *prev = (m == 2) ? v0 : out;
    sk_step_kernel<false><<<grid, kSkThreads, 0, st>>>(n, slice_ptr, col, geom, total, on, x, prev, out,
                                                       partial + (size_t)(2 * (m - 1)) * ps, ps, two_over_a, shift);
    TB_CHECK_LAUNCH();
  }
  moment_reduce_kernel<<<(M + 255) / 256, 256, 0, st>>>(partial, grid, 1, M, 1.0 / (double)(n * kNO), 1, 1.0 + 1e-6,
                                                        mu_out, flags);
  TB_CHECK_LAUNCH();
  if (ms_out) TB_CUDA(cudaEventRecord(ev[1], st));
  int hflags[4] = {0, 0, 0, 0};
  TB_CUDA(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
  TB_CUDA(cudaStreamSynchronize(st));
  if (ms_out) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    *ms_out = ms;
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
  }
  if (hflags[0] & 2) return fail(TB_ERR_NOT_FINITE, "sk_kpm_moments: non-finite moment");
  if (hflags[0] & 1)
    return fail(TB_ERR_BOUNDS, "sk_kpm_moments: |mu_n| > 1 + 1e-6; the spectrum is not inside [b - a, b + a]");
  return TB_OK;
}
