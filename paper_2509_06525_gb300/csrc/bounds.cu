// FP64 spectral bounds for the Chebyshev rescaling H~ = (H - b)/a of the
// KPM/LSQT method (arXiv 2509.06525 Sec. 2.4).
//
//  * Gershgorin: [min_i(eps_i - R_i), max_i(eps_i + R_i)], R_i = sum_j |H_ij|.
//  * Lanczos: k steps of the symmetric three-term recurrence (FP64, no
//    reorthogonalisation) from q_i = u(seed, 0, i) - 1/2, normalised, with
//    u the SplitMix64 counter deviate of the KPM random phases.  The
//    extreme eigenvalues of the tridiagonal T_k come from Sturm-sequence
//    multisection: each of the 32 lanes of one warp counts eigenvalues
//    below its own trial point, so every round narrows the bracket 32-fold.
//  * delta = 0.01 (theta_max - theta_min); E_max = min(G_max, theta_max +
//    delta), E_min = max(G_min, theta_min - delta); a = (E_max - E_min) /
//    (2 - 0.01), b = (E_max + E_min) / 2.
// Every reduction is two-level (CTA partials, then one CTA in fixed order),
// so the result is bitwise reproducible.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace gputb {
namespace {

constexpr int kB = 256;

__device__ __forceinline__ uint64_t smix(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__device__ __forceinline__ T block_sum(T v) {
  __shared__ T sh[kB / 32];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kB / 32; ++w) s += sh[w];
  __syncthreads();
  return s;  // valid in thread 0
}

__device__ __forceinline__ void block_minmax(double lo, double hi, double *out_lo, double *out_hi) {
  __shared__ double sl[kB / 32], sh[kB / 32];
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
    double a = sl[0], b = sh[0];
    for (int w = 1; w < kB / 32; ++w) {
      a = fmin(a, sl[w]);
      b = fmax(b, sh[w]);
    }
    *out_lo = a;
    *out_hi = b;
  }
}

template <typename valT>
__global__ void gershgorin_kernel(int64_t n, const int64_t *__restrict__ sp, const int32_t *__restrict__ col,
                                  const valT *__restrict__ val, const valT *__restrict__ diag,
                                  double *__restrict__ part_lo, double *__restrict__ part_hi) {
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x; i < n; i += (int64_t)gridDim.x * kB) {
    const int64_t sb = sp[i >> 5];
    const int w = static_cast<int>((sp[(i >> 5) + 1] - sb) >> 5);
    double r = 0.0;
    if constexpr (sizeof(valT) == 4) {
      // FP32 values: the row sum as an FP32 pair (TwoSum per term; about 47
      // bits), one conversion to FP64 per row instead of one per element
      float rh = 0.0f, rl = 0.0f;
      for (int s = 0; s < w; ++s) {
        const float a = fabsf(val[sb + (i & 31) + 32 * s]);
        const float t = rh + a;
        const float bb = t - rh;
        rl += (rh - (t - bb)) + (a - bb);
        rh = t;
      }
      r = (double)rh + (double)rl;
    } else {
      for (int s = 0; s < w; ++s) r += fabs((double)val[sb + (i & 31) + 32 * s]);
    }
    const double d = diag ? (double)diag[i] : 0.0;
    lo = fmin(lo, d - r);
    hi = fmax(hi, d + r);
  }
  block_minmax(lo, hi, part_lo + blockIdx.x, part_hi + blockIdx.x);
}

__global__ void lanczos_start_kernel(int64_t n, uint64_t seed, double *__restrict__ q, double *__restrict__ part) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x; i < n; i += (int64_t)gridDim.x * kB) {
    const uint64_t z = smix(seed ^ smix((0ull << 32) + (uint64_t)i));
    const double v = static_cast<double>(z >> 11) * 0x1.0p-53 - 0.5;
    q[i] = v;
    acc = fma(v, v, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// scal[slot] = sum of partials (fixed order); mode 1: sqrt
__global__ void reduce_scalar_kernel(const double *__restrict__ part, int nparts, double *__restrict__ scal,
                                     int slot, int mode) {
  double acc = 0.0;
  for (int c = threadIdx.x; c < nparts; c += kB) acc += part[c];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) scal[slot] = mode == 1 ? sqrt(s) : s;
}

__global__ void scale_kernel(int64_t n, double *__restrict__ q, const double *__restrict__ norm) {
  const double inv = 1.0 / norm[0];
  for (int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x; i < n; i += (int64_t)gridDim.x * kB) q[i] *= inv;
}

// w = H q - beta_prev q_prev; part = sum q.w.  A row with at most 16 slots
// issues all its column and value loads before its gathers (memory-level
// parallelism: the kernel is bound by latency, not by its FP64 arithmetic).
template <typename valT>
__global__ void __launch_bounds__(kB) lanczos_spmv_kernel(int64_t n, const int64_t *__restrict__ sp,
                                                          const int32_t *__restrict__ col,
                                                          const valT *__restrict__ val, const valT *__restrict__ diag,
                                                          const double *__restrict__ q,
                                                          const double *__restrict__ qprev,
                                                          const double *__restrict__ beta_prev,
                                                          double *__restrict__ w, double *__restrict__ part) {
  constexpr int kW = 16;
  const double bp = beta_prev ? *beta_prev : 0.0;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x; i < n; i += (int64_t)gridDim.x * kB) {
    const int64_t sb = __ldg(sp + (i >> 5));
    const int ww = static_cast<int>((__ldg(sp + (i >> 5) + 1) - sb) >> 5);
    const int64_t e0 = sb + (i & 31);
    const double qi = __ldg(q + i);
    const double qp = qprev ? __ldcs(qprev + i) : 0.0;
    double y = diag ? (double)__ldg(diag + i) * qi : 0.0;
    if (ww <= kW) {
      int32_t j[kW];
      double h[kW];
#pragma unroll
      for (int s = 0; s < kW; ++s)
        if (s < ww) {
          j[s] = __ldcs(col + e0 + 32 * s);
          h[s] = (double)__ldcs(val + e0 + 32 * s);
        }
#pragma unroll
      for (int s = 0; s < kW; ++s)
        if (s < ww) y = fma(h[s], __ldg(q + j[s]), y);
    } else {
      for (int s = 0; s < ww; ++s) {
        const int64_t e = e0 + 32 * s;
        y = fma((double)val[e], __ldg(q + col[e]), y);
      }
    }
    if (qprev) y = fma(-bp, qp, y);
    w[i] = y;
    acc = fma(qi, y, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// w -= alpha q; part = sum w.w
__global__ void lanczos_orth_kernel(int64_t n, const double *__restrict__ q, const double *__restrict__ alpha,
                                    double *__restrict__ w, double *__restrict__ part) {
  const double a = *alpha;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x; i < n; i += (int64_t)gridDim.x * kB) {
    const double v = fma(-a, q[i], w[i]);
    w[i] = v;
    acc = fma(v, v, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// ---- Lanczos for an FP32 Hamiltonian in double-float arithmetic ----------
// GB300 issues FP64 at a small fraction of its FP32 rate, and an FP64 SpMV of
// an FP32 matrix spends a conversion and an FMA on that pipe per stored
// element.  For FP32 values the vectors are kept as unevaluated sums
// hi + lo of two floats (about 48 significant bits) and every product and
// sum is made from the error-free transformations TwoSum (Knuth) and
// TwoProduct (Dekker, in its FMA form): a + b = s + e and a * b = p + e hold
// exactly in round-to-nearest FP32.  The Lanczos vectors are stored
// unnormalised, U_j, with q_j = s_j U_j and s_j = 1 / beta_{j-1} applied on
// read, so no separate scaling pass is needed and w overwrites U_{j-1}.
struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ dfl fast_two_sum(float a, float b) {  // needs |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  dfl s = two_sum(a.hi, b.hi);
  const dfl t = two_sum(a.lo, b.lo);
  s = fast_two_sum(s.hi, s.lo + t.hi);
  return fast_two_sum(s.hi, s.lo + t.lo);
}

// products that feed TwoSum use __fmul_rn, which the compiler never contracts
// into an FMA (a contracted sum would break the error-free identities)
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}

__device__ __forceinline__ dfl to_dfl(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - (double)hi)};
}

__device__ __forceinline__ double to_double(dfl a) { return (double)a.hi + (double)a.lo; }

// running sum S += h * (u.hi + u.lo): S.hi collects the rounded products
// exactly (TwoSum), S.lo the rounding errors and the low-order products
__device__ __forceinline__ void df_axpy_acc(float h, float2 u, float &shi, float &slo) {
  const float p = __fmul_rn(h, u.x);
  const float e = fmaf(h, u.x, -p);
  const dfl t = two_sum(shi, p);
  shi = t.hi;
  slo += t.lo + fmaf(h, u.y, e);
}

__global__ void lanczos_start_df_kernel(int64_t n, uint64_t seed, float2 *__restrict__ u,
                                        double *__restrict__ part) {
  dfl acc{0.0f, 0.0f};
  for (int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x; i < n; i += (int64_t)gridDim.x * kB) {
    const uint64_t z = smix(seed ^ smix((0ull << 32) + (uint64_t)i));
    const dfl v = to_dfl(static_cast<double>(z >> 11) * 0x1.0p-53 - 0.5);
    u[i] = make_float2(v.hi, v.lo);
    acc = df_add(acc, df_mul(v, v));
  }
  const double s = block_sum(to_double(acc));
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// w = s_j H U_j - beta_{j-1} s_{j-1} U_{j-1}, written over U_{j-1} (each row
// is read and written by the same thread); part = sum (s_j U_j) . w
template <bool PREV>
__global__ void __launch_bounds__(kB, 3) lanczos_spmv_df_kernel(
    int64_t n, const int64_t *__restrict__ sp, const int32_t *__restrict__ col, const float *__restrict__ val,
    const float *__restrict__ diag, const float2 *__restrict__ u, const double *__restrict__ s_j, float2 *prev_w,
    const double *__restrict__ s_prev, const double *__restrict__ beta_prev, double *__restrict__ part) {
  constexpr int kW = 16;
  const dfl sj = to_dfl(*s_j);
  const dfl c = PREV ? to_dfl(-(*beta_prev) * (*s_prev)) : dfl{0.0f, 0.0f};
  dfl acc{0.0f, 0.0f};
  for (int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x; i < n; i += (int64_t)gridDim.x * kB) {
    const int64_t sb = __ldg(sp + (i >> 5));
    const int ww = static_cast<int>((__ldg(sp + (i >> 5) + 1) - sb) >> 5);
    const int64_t e0 = sb + (i & 31);
    const float2 ui = __ldg(u + i);
    float2 pv = make_float2(0.0f, 0.0f);
    if (PREV) pv = __ldcs(prev_w + i);
    float shi = 0.0f, slo = 0.0f;
    if (diag) df_axpy_acc(__ldg(diag + i), ui, shi, slo);
    if (ww <= kW) {
      int32_t j[kW];
      float h[kW];
#pragma unroll
      for (int s = 0; s < kW; ++s)
        if (s < ww) {
          j[s] = __ldcs(col + e0 + 32 * s);
          h[s] = __ldcs(val + e0 + 32 * s);
        }
#pragma unroll
      for (int s = 0; s < kW; ++s)
        if (s < ww) df_axpy_acc(h[s], __ldg(u + j[s]), shi, slo);
    } else {
      for (int s = 0; s < ww; ++s) {
        const int64_t e = e0 + 32 * s;
        df_axpy_acc(val[e], __ldg(u + col[e]), shi, slo);
      }
    }
    dfl y = df_mul(two_sum(shi, slo), sj);
    if (PREV) y = df_add(y, df_mul(dfl{pv.x, pv.y}, c));
    prev_w[i] = make_float2(y.hi, y.lo);
    acc = df_add(acc, df_mul(df_mul(dfl{ui.x, ui.y}, sj), y));
  }
  const double s = block_sum(to_double(acc));
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// w -= alpha_j s_j U_j; part = sum w.w
__global__ void lanczos_orth_df_kernel(int64_t n, const float2 *__restrict__ u, const double *__restrict__ s_j,
                                       const double *__restrict__ alpha, float2 *__restrict__ w,
                                       double *__restrict__ part) {
  const dfl c = to_dfl(-(*alpha) * (*s_j));
  dfl acc{0.0f, 0.0f};
  for (int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x; i < n; i += (int64_t)gridDim.x * kB) {
    const float2 a = __ldg(u + i), b = w[i];
    const dfl v = df_add(dfl{b.x, b.y}, df_mul(dfl{a.x, a.y}, c));
    w[i] = make_float2(v.hi, v.lo);
    acc = df_add(acc, df_mul(v, v));
  }
  const double s = block_sum(to_double(acc));
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// beta = sqrt(sum of partials) (skipped when beta is null), inv = 1 / beta
__global__ void reduce_norm_kernel(const double *__restrict__ part, int nparts, double *__restrict__ beta,
                                   double *__restrict__ inv) {
  double acc = 0.0;
  for (int c = threadIdx.x; c < nparts; c += kB) acc += part[c];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) {
    const double r = sqrt(s);
    if (beta) *beta = r;
    *inv = 1.0 / r;
  }
}

__device__ int sturm_below(const double *alpha, const double *beta, int m, double x) {
  int count = 0;
  double d = 1.0;
  for (int i = 0; i < m; ++i) {
    d = (alpha[i] - x) - (i > 0 ? beta[i - 1] * beta[i - 1] / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++count;
  }
  return count;
}

// One warp: extremes of tridiag(alpha[0..m), beta[0..m-1)) by 32-way
// multisection, then the bounds combination.  out = {emin, emax, a, b}.
__global__ void finish_bounds_kernel(const double *__restrict__ alpha, const double *__restrict__ beta, int m,
                                     const double *__restrict__ g_lo_part, const double *__restrict__ g_hi_part,
                                     int nparts, double margin, double eps, double *__restrict__ out) {
  __shared__ double sa[1024], sb[1024];
  const int lane = threadIdx.x;
  for (int k = lane; k < m; k += 32) sa[k] = alpha[k];
  for (int k = lane; k < m - 1; k += 32) sb[k] = beta[k];
  double glo = INFINITY, ghi = -INFINITY;
  for (int c = lane; c < nparts; c += 32) {
    glo = fmin(glo, g_lo_part[c]);
    ghi = fmax(ghi, g_hi_part[c]);
  }
  for (int off = 16; off > 0; off >>= 1) {
    glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, off));
    ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, off));
  }
  __syncwarp();
  // Gershgorin interval of T as the initial bracket
  double tlo = INFINITY, thi = -INFINITY;
  for (int k = lane; k < m; k += 32) {
    double r = 0.0;
    if (k > 0) r += fabs(sb[k - 1]);
    if (k < m - 1) r += fabs(sb[k]);
    tlo = fmin(tlo, sa[k] - r);
    thi = fmax(thi, sa[k] + r);
  }
  for (int off = 16; off > 0; off >>= 1) {
    tlo = fmin(tlo, __shfl_xor_sync(0xffffffffu, tlo, off));
    thi = fmax(thi, __shfl_xor_sync(0xffffffffu, thi, off));
  }
  double ext[2];
  for (int which = 0; which < 2; ++which) {
    // smallest eigenvalue: count(x) >= 1; largest: count(x) >= m
    const int target = which == 0 ? 1 : m;
    double lo = tlo, hi = thi;
    for (int round = 0; round < 40; ++round) {
      const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
      const bool ok = sturm_below(sa, sb, m, x) >= target;
      const unsigned mask = __ballot_sync(0xffffffffu, ok);
      // first lane whose point already has >= target eigenvalues below it
      const int first = mask ? __ffs(mask) - 1 : 32;
      const double nlo = first == 0 ? lo : lo + (hi - lo) * (double)first / 33.0;
      const double nhi = first == 32 ? hi : lo + (hi - lo) * (double)(first + 1) / 33.0;
      if (!(nhi - nlo < hi - lo)) break;
      lo = nlo;
      hi = nhi;
    }
    ext[which] = 0.5 * (lo + hi);
  }
  if (lane == 0) {
    const double tmin = ext[0], tmax = ext[1];
    const double delta = margin * (tmax - tmin);
    const double emax = fmin(ghi, tmax + delta);
    const double emin = fmax(glo, tmin - delta);
    out[0] = emin;
    out[1] = emax;
    out[2] = (emax - emin) / (2.0 - eps);
    out[3] = 0.5 * (emax + emin);
    out[4] = tmin;
    out[5] = tmax;
    out[6] = glo;
    out[7] = ghi;
  }
}

int grid_for(int64_t n) {
  const int64_t need = (n + kB - 1) / kB;
  const int64_t cap = (int64_t)sm_count() * 8;
  return static_cast<int>(need < cap ? need : cap);
}

template <typename valT>
tb_status run_bounds(int64_t n, const int64_t *sp, const int32_t *col, const valT *val, const valT *diag, int k,
                     uint64_t seed, double *out_host, void *ws, size_t wsb, cudaStream_t st) {
  const int grid = grid_for(n);
  Carver cv(ws, wsb);
  double *q0 = cv.take<double>(n), *q1 = cv.take<double>(n), *w = cv.take<double>(n);
  double *part = cv.take<double>(grid), *glo = cv.take<double>(grid), *ghi = cv.take<double>(grid);
  double *alpha = cv.take<double>(k), *beta = cv.take<double>(k), *norm = cv.take<double>(1);
  double *out = cv.take<double>(8), *inv = cv.take<double>(k + 1);
  if (!cv.ok()) return fail(TB_ERR_WORKSPACE, "tb_spectral_bounds: workspace too small");
  gershgorin_kernel<valT><<<grid, kB, 0, st>>>(n, sp, col, val, diag, glo, ghi);
  TB_CHECK_LAUNCH();
  if constexpr (sizeof(valT) == 4) {
    // double-float Lanczos on two buffers of float2 (inside q0 and q1)
    float2 *ua = reinterpret_cast<float2 *>(q0), *ub = reinterpret_cast<float2 *>(q1);
    // one wave of resident CTAs for the SpMV (its grid-stride loop has no tail wave)
    static int per_sm = 0;
    if (per_sm == 0 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lanczos_spmv_df_kernel<true>, kB,
                                                                      0) != cudaSuccess ||
                        per_sm <= 0))
      per_sm = 3;
    const int gs = std::min<int64_t>(grid, (int64_t)per_sm * sm_count());
    lanczos_start_df_kernel<<<grid, kB, 0, st>>>(n, seed, ua, part);
    TB_CHECK_LAUNCH();
    reduce_norm_kernel<<<1, kB, 0, st>>>(part, grid, nullptr, inv);
    TB_CHECK_LAUNCH();
    for (int j = 0; j < k; ++j) {
      if (j == 0)
        lanczos_spmv_df_kernel<false><<<gs, kB, 0, st>>>(n, sp, col, val, diag, ua, inv, ub, nullptr, nullptr,
                                                         part);
      else
        lanczos_spmv_df_kernel<true><<<gs, kB, 0, st>>>(n, sp, col, val, diag, ua, inv + j, ub, inv + j - 1,
                                                        beta + j - 1, part);
      TB_CHECK_LAUNCH();
      reduce_scalar_kernel<<<1, kB, 0, st>>>(part, gs, alpha, j, 0);
      TB_CHECK_LAUNCH();
      if (j == k - 1) break;
      lanczos_orth_df_kernel<<<grid, kB, 0, st>>>(n, ua, inv + j, alpha + j, ub, part);
      TB_CHECK_LAUNCH();
      reduce_norm_kernel<<<1, kB, 0, st>>>(part, grid, beta + j, inv + j + 1);
      TB_CHECK_LAUNCH();
      float2 *t = ua;  // U_{j+1} = w; U_j becomes the previous vector
      ua = ub;
      ub = t;
    }
  } else {
    lanczos_start_kernel<<<grid, kB, 0, st>>>(n, seed, q1, part);
    TB_CHECK_LAUNCH();
    reduce_scalar_kernel<<<1, kB, 0, st>>>(part, grid, norm, 0, 1);
    TB_CHECK_LAUNCH();
    scale_kernel<<<grid, kB, 0, st>>>(n, q1, norm);
    TB_CHECK_LAUNCH();
    double *q = q1, *qprev = q0;
    for (int j = 0; j < k; ++j) {
      lanczos_spmv_kernel<valT><<<grid, kB, 0, st>>>(n, sp, col, val, diag, q, j > 0 ? qprev : nullptr,
                                                     j > 0 ? beta + (j - 1) : nullptr, w, part);
      TB_CHECK_LAUNCH();
      reduce_scalar_kernel<<<1, kB, 0, st>>>(part, grid, alpha, j, 0);
      TB_CHECK_LAUNCH();
      if (j == k - 1) break;
      lanczos_orth_kernel<<<grid, kB, 0, st>>>(n, q, alpha + j, w, part);
      TB_CHECK_LAUNCH();
      reduce_scalar_kernel<<<1, kB, 0, st>>>(part, grid, beta, j, 1);
      TB_CHECK_LAUNCH();
      // q_{j+1} = w / beta_j, written over q_{j-1}
      scale_kernel<<<grid, kB, 0, st>>>(n, w, beta + j);
      double *t = qprev;
      qprev = q;
      q = w;
      w = t;
      TB_CHECK_LAUNCH();
    }
  }
  finish_bounds_kernel<<<1, 32, 0, st>>>(alpha, beta, k, glo, ghi, grid, 0.01, 0.01, out);
  TB_CHECK_LAUNCH();
  TB_CUDA(cudaMemcpyAsync(out_host, out, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
  TB_CUDA(cudaStreamSynchronize(st));
  for (int c = 0; c < 4; ++c)
    if (!std::isfinite(out_host[c])) return fail(TB_ERR_NOT_FINITE, "tb_spectral_bounds: non-finite bound");
  if (!(out_host[2] > 0.0)) return fail(TB_ERR_NOT_FINITE, "tb_spectral_bounds: degenerate spectrum (a <= 0)");
  return TB_OK;
}

}  // namespace
}  // namespace gputb

using namespace gputb;

extern "C" size_t tb_spectral_bounds_workspace_size(int64_t n, int32_t lanczos_steps) {
  if (n <= 0 || lanczos_steps < 1) return 0;
  Carver cv(nullptr, 0);
  const int grid = grid_for(n);
  cv.take<double>(n);
  cv.take<double>(n);
  cv.take<double>(n);
  cv.take<double>(grid);
  cv.take<double>(grid);
  cv.take<double>(grid);
  cv.take<double>(lanczos_steps);
  cv.take<double>(lanczos_steps);
  cv.take<double>(1);
  cv.take<double>(8);
  cv.take<double>(lanczos_steps + 1);
  return cv.used + 256;
}

extern "C" tb_status tb_spectral_bounds(int64_t n, const int64_t *slice_ptr, const int32_t *col, const void *val,
                                        const void *diag, int32_t precision, int32_t lanczos_steps, uint64_t seed,
                                        double *bounds_out, void *workspace, size_t workspace_bytes, void *stream) {
  TB_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "tb_spectral_bounds: bad n");
  TB_REQUIRE(lanczos_steps >= 2 && lanczos_steps <= 1024 && lanczos_steps <= n,
             "tb_spectral_bounds: lanczos_steps must be in [2, min(1024, n)]");
  TB_REQUIRE(slice_ptr && bounds_out && workspace, "tb_spectral_bounds: null pointer argument");
  TB_REQUIRE(precision == TB_F32 || precision == TB_F64, "tb_spectral_bounds: bad precision");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (precision == TB_F32)
    return run_bounds<float>(n, slice_ptr, col, static_cast<const float *>(val), static_cast<const float *>(diag),
                             lanczos_steps, seed, bounds_out, workspace, workspace_bytes, st);
  return run_bounds<double>(n, slice_ptr, col, static_cast<const double *>(val), static_cast<const double *>(diag),
                            lanczos_steps, seed, bounds_out, workspace, workspace_bytes, st);
}
