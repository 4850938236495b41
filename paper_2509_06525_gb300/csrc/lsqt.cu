// Velocity-autocorrelation (VAC) conductivity of the LSQT method,
// Eq. 3 (sigma) of arXiv 2509.06525, Sec. 2.4:
//   sigma(E, t) = (2 e^2 / Omega) int_0^t Tr[delta(E - H) Re(V V(tau))] dtau.
//
// * velocity   V = (i/hbar)[H, X]: V_ij = (i/hbar) (x_j - x_i) H_ij, stored as
//              the real SELL values vval_e = H_ij (d_ij . e) of the matrix
//              pattern (d_ij the minimum-image bond vector, e the direction).
// * trace      Tr[delta V U^+ V U] ~ <phi_L(tau)| V delta(E - H) |phi_R(tau)>
//              over random-phase vectors, phi_L(0) = V phi, phi_R(0) = phi,
//              both propagated by U(dt) = exp(-i H dt / hbar).
// * moments    mu_n(tau) = Re <V phi_L| T_n(H~) |phi_R> / N: the Chebyshev
//              recursion of the KPM step kernels started from phi_R, with
//              w = V phi_L as the dot vector (kpm_step.cuh); mu_0 comes from
//              the velocity kernel that forms w.
// * time step  exp(-i x H~) = sum_k eps_k (-i)^k J_k(x) T_k(H~), x = a dt /
//              hbar (Jacobi-Anger; eps_0 = 1, eps_k = 2), times the phase
//              exp(-i b dt / hbar); the series is cut where |J_k(x)| < 1e-17
//              and k > x.  One fused kernel per term: the Chebyshev step
//              plus the complex update acc += c_k T_k(H~) phi.
// * energy     C(E, tau) and S(E, t) = int_0^t C dtau from the moments by the
//              damped Chebyshev series of the DOS and the trapezoid rule.
#include <cmath>
#include <vector>

#include "geometry.cuh"
#include "kpm_step.cuh"

namespace gputb {
namespace {

constexpr double kHbar = 0.6582119569;   // eV fs (CODATA 2018)

// vval_e = val_e (d_ij . dir); phantom rows 0
template <typename valT>
__global__ void velocity_values_kernel(const double *__restrict__ pos, int64_t n, int64_t n_slices, Box B,
                                       const int64_t *__restrict__ sp, const int32_t *__restrict__ col,
                                       const valT *__restrict__ val, double ex, double ey, double ez,
                                       valT *__restrict__ vval) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_slices * 32) return;
  const int64_t sb = sp[i >> 5];
  const int w = static_cast<int>((sp[(i >> 5) + 1] - sb) >> 5);
  int64_t e = sb + (i & 31);
  for (int s = 0; s < w; ++s, e += 32) {
    double v = 0.0;
    if (i < n) {
      const int32_t j = col[e];
      if (j != i) {
        const double3 d = bond_vector(B, pos, i, j);
        v = (double)val[e] * (d.x * ex + d.y * ey + d.z * ez);
      }
    }
    vval[e] = static_cast<valT>(v);
  }
}

// out = (i/hbar) sum_j vval_ij x_j; with z, also the CTA partials of
// Re <out|z> (mu_0 of the VAC moments) into partial[cta][r]
template <typename real, typename valT, int R, int CPT, bool DOT>
__global__ void __launch_bounds__(kBlock) velocity_apply_kernel(int64_t n, const int64_t *__restrict__ sp,
                                                                const int32_t *__restrict__ col,
                                                                const valT *__restrict__ vval,
                                                                const real *__restrict__ x, const real *__restrict__ z,
                                                                real *__restrict__ out, double *__restrict__ partial,
                                                                real inv_hbar) {
  constexpr int TPR = R / CPT;
  constexpr int RPB = kBlock / TPR;
  const int part = threadIdx.x % TPR;
  DotAcc<real> acc[CPT];
  const int64_t nblk = (n + RPB - 1) / RPB;
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int64_t i = blk * RPB + threadIdx.x / TPR;
    if (i >= n) continue;
    const int64_t sb = __ldg(sp + (i >> 5));
    const int w = static_cast<int>((__ldg(sp + (i >> 5) + 1) - sb) >> 5);
    real y[2 * CPT];
#pragma unroll
    for (int c = 0; c < 2 * CPT; ++c) y[c] = real(0);
    int64_t e = sb + (i & 31);
    for (int s = 0; s < w; ++s, e += 32) {
      const int32_t j = __ldg(col + e);
      const real h = static_cast<real>(__ldg(vval + e));
      real xv[2 * CPT];
      ld_gather<real, CPT>(x + ((int64_t)j * R + part * CPT) * 2, xv);
#pragma unroll
      for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(h, xv[c], y[c]);
    }
    real o[2 * CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {   // i (a + i b) = -b + i a
      o[2 * c] = -inv_hbar * y[2 * c + 1];
      o[2 * c + 1] = inv_hbar * y[2 * c];
    }
    const int64_t off = (i * R + part * CPT) * 2;
    st_stream<real, CPT>(out + off, o);
    if (DOT) {
      real zz[2 * CPT];
      ld_stream<real, CPT>(z + off, zz);
#pragma unroll
      for (int c = 0; c < CPT; ++c) acc[c].add(o[2 * c], o[2 * c + 1], zz[2 * c], zz[2 * c + 1]);
    }
  }
  if (DOT) {
    double sum[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) sum[c] = acc[c].value();
    cta_partial<R, CPT>(sum, partial + (int64_t)blockIdx.x * R);
  }
}

// One term of the propagator series.  FIRST: t1 = H~ x -> io, acc = c0 x + c1 t1;
// else: t_{k+1} = 2 H~ x - t_{k-1} written over io (which holds t_{k-1}),
// acc += c t_{k+1}.  H~ x = alpha_0 (sum_s val x[col] + (diag_i - shift) x_i)
// with alpha = 1/a (FIRST) or 2/a.
// register budget of the propagation kernel: 4 resident CTAs (64 registers)
// with one FP32 complex number per thread, 3 for FP32 with more, 2 for FP64
template <typename real, int R, int CPT>
constexpr int propagate_min_blocks() {
  return sizeof(real) == 8 ? 2 : (R == 1 ? 4 : (CPT >= 4 ? 2 : 3));
}

template <typename real, typename valT, int R, int CPT, bool FIRST>
__global__ void __launch_bounds__(kBlock, propagate_min_blocks<real, R, CPT>()) propagate_term_kernel(
    int64_t n, const int64_t *__restrict__ sp, const int32_t *__restrict__ col, const valT *__restrict__ val,
    const valT *__restrict__ diag, const real *__restrict__ x, real *io, real *__restrict__ acc, real alpha,
    real shift, real c0r, real c0i, real cr, real ci) {
  constexpr int TPR = R / CPT;
  constexpr int RPB = kBlock / TPR;
  const int part = threadIdx.x % TPR;
  const int64_t nblk = (n + RPB - 1) / RPB;
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int64_t i = blk * RPB + threadIdx.x / TPR;
    if (i >= n) continue;
    const int64_t off = (i * R + part * CPT) * 2;
    real p[2 * CPT], a[2 * CPT];
    if (!FIRST) {
      ld_stream<real, CPT>(io + off, p);
      ld_stream<real, CPT>(acc + off, a);
    }
    const real d = (diag ? static_cast<real>(__ldg(diag + i)) : real(0)) - shift;
    const int64_t sb = __ldg(sp + (i >> 5));
    const int w = static_cast<int>((__ldg(sp + (i >> 5) + 1) - sb) >> 5);
    const int64_t e0 = sb + (i & 31);
    real y[2 * CPT];
#pragma unroll
    for (int c = 0; c < 2 * CPT; ++c) y[c] = real(0);
    if (w <= kFastW) {
      int32_t j[kFastW];
      real h[kFastW];
#pragma unroll
      for (int s = 0; s < kFastW; ++s)
        if (s < w) {
          j[s] = __ldcs(col + e0 + 32 * s);
          h[s] = static_cast<real>(__ldcs(val + e0 + 32 * s));
        }
#pragma unroll
      for (int s = 0; s < kFastW; ++s)
        if (s < w) {
          real xv[2 * CPT];
          ld_gather<real, CPT>(x + ((int64_t)j[s] * R + part * CPT) * 2, xv);
#pragma unroll
          for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(h[s], xv[c], y[c]);
        }
    } else {
      int64_t e = e0;
      for (int s = 0; s < w; ++s, e += 32) {
        const int32_t jj = __ldcs(col + e);
        const real hh = static_cast<real>(__ldcs(val + e));
        real xv[2 * CPT];
        ld_gather<real, CPT>(x + ((int64_t)jj * R + part * CPT) * 2, xv);
#pragma unroll
        for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(hh, xv[c], y[c]);
      }
    }
    real xi[2 * CPT];
    ld_gather<real, CPT>(x + off, xi);
#pragma unroll
    for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(d, xi[c], y[c]);
    real o[2 * CPT];
#pragma unroll
    for (int c = 0; c < 2 * CPT; ++c) o[c] = FIRST ? alpha * y[c] : fma(alpha, y[c], -p[c]);
    st_stream<real, CPT>(io + off, o);
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const real orr = o[2 * c], oi = o[2 * c + 1];
      real ar, ai;
      if (FIRST) {
        ar = c0r * xi[2 * c] - c0i * xi[2 * c + 1];
        ai = c0r * xi[2 * c + 1] + c0i * xi[2 * c];
      } else {
        ar = a[2 * c];
        ai = a[2 * c + 1];
      }
      a[2 * c] = ar + (cr * orr - ci * oi);
      a[2 * c + 1] = ai + (cr * oi + ci * orr);
    }
    st_stream<real, CPT>(acc + off, a);
  }
}

// phi[i, r] = exp(2 pi i u(seed, r0 + r, i)) (the KPM random phases)
template <typename real, int R>
__global__ void lsqt_phase_kernel(int64_t n, uint64_t seed, int64_t r0, real *__restrict__ phi) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * R) return;
  const int64_t i = t / R;
  const int r = static_cast<int>(t % R);
  real sn, co;
  phase_cis<real>(seed, (uint64_t)(r0 + r), (uint64_t)i, co, sn);
  phi[2 * t] = co;
  phi[2 * t + 1] = sn;
}

// coef[j][n] = g_n (2 - delta_n0) mean_r mu[j][r][n]
__global__ void vac_coef_kernel(const double *__restrict__ mu, int n_times, int R, int M, int kernel, double lam,
                                double *__restrict__ coef) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n_times * M) return;
  const int j = static_cast<int>(t / M), m = static_cast<int>(t % M);
  double g = 1.0;
  if (kernel == TB_KERNEL_JACKSON) {
    const double q = M_PI / (M + 1);
    g = ((M - m + 1) * cos(q * m) + sin(q * m) * cos(q) / sin(q)) / (M + 1);
  } else if (kernel == TB_KERNEL_LORENTZ) {
    g = sinh(lam * (1.0 - (double)m / M)) / sinh(lam);
  }
  double s = 0.0;
  for (int r = 0; r < R; ++r) s += mu[((int64_t)j * R + r) * M + m];
  coef[t] = g * (m == 0 ? 1.0 : 2.0) * s / R;
}

// C[j][k] = sum_n coef[j][n] T_n(x_k) / (pi a sqrt(1 - x_k^2)), S[j][k] its
// running trapezoid integral over j (S[0] = 0)
__global__ void vac_series_kernel(const double *__restrict__ coef, int n_times, int M, double a, double b,
                                  const double *__restrict__ energy, int K, double dt, double *__restrict__ corr,
                                  double *__restrict__ sig) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double x = (energy[k] - b) / a;
  const bool inside = fabs(x) < 1.0;
  const double w = inside ? 1.0 / (M_PI * a * sqrt(1.0 - x * x)) : 0.0;
  double s_run = 0.0, c_prev = 0.0;
  for (int j = 0; j < n_times; ++j) {
    const double *c = coef + (int64_t)j * M;
    double val = 0.0;
    if (inside) {
      double t0 = 1.0, t1 = x, acc = c[0];
      if (M > 1) acc += c[1] * x;
      for (int m = 2; m < M; ++m) {
        const double t2 = 2.0 * x * t1 - t0;
        acc += c[m] * t2;
        t0 = t1;
        t1 = t2;
      }
      val = acc * w;
    }
    if (j > 0) s_run += 0.5 * dt * (c_prev + val);
    corr[(int64_t)j * K + k] = val;
    if (sig) sig[(int64_t)j * K + k] = s_run;
    c_prev = val;
  }
}

template <typename real, typename valT, int R>
struct LsqtRunner {
  using Kit = StepKit<real, valT, R>;
  static constexpr int CPT = Kit::CPT;
  static constexpr int kVectors = 7;   // phi_L, phi_R, w, A, B, X1, ACC

  static int64_t padded_rows(int64_t n) { return (n + Kit::kRowPad - 1) / Kit::kRowPad * Kit::kRowPad; }

  static size_t workspace(int64_t n, int M) {
    Carver cv(nullptr, 0);
    for (int k = 0; k < kVectors; ++k) cv.take<real>((size_t)padded_rows(n) * R * 2);
    cv.take<double>((size_t)(M + 1) * Kit::max_grid(n) * R);
    cv.take<int>(4);
    if (Kit::any_banded()) {
      cv.take<BandRec>(Kit::plan_records(n));
      cv.take<uint16_t>((size_t)padded_rows(n) * kBandSlots);
    }
    return cv.used + 256;
  }

  // c_k = exp(-i b dt/hbar) eps_k (-i)^k J_k(a dt/hbar), k = 0 .. K
  static void propagator_coefficients(double a, double b, double dt, std::vector<double> &cr,
                                      std::vector<double> &ci) {
    const double x = a * dt / kHbar;
    const double ph = -b * dt / kHbar;
    const double pr = std::cos(ph), pi = std::sin(ph);
    cr.clear();
    ci.clear();
    for (int k = 0; k < 1000; ++k) {
      const double jk = std::cyl_bessel_j((double)k, x);
      if (k > x + 2 && std::fabs(jk) < 1e-17) break;
      const double mag = (k == 0 ? 1.0 : 2.0) * jk;
      // (-i)^k = 1, -i, -1, i
      double qr = 0.0, qi = 0.0;
      switch (k & 3) {
        case 0: qr = mag; break;
        case 1: qi = -mag; break;
        case 2: qr = -mag; break;
        default: qi = mag; break;
      }
      cr.push_back(pr * qr - pi * qi);
      ci.push_back(pr * qi + pi * qr);
    }
  }

  static tb_status propagate(int grid, int64_t n, const int64_t *sp, const int32_t *col, const valT *val,
                             const valT *diag, real *&phi, real *x1, real *&acc, real inv_a, real two_over_a,
                             real shift, const std::vector<double> &cr, const std::vector<double> &ci,
                             cudaStream_t st) {
    const int K = (int)cr.size();
    const real c1r = K > 1 ? (real)cr[1] : real(0), c1i = K > 1 ? (real)ci[1] : real(0);
    propagate_term_kernel<real, valT, R, CPT, true><<<grid, kBlock, 0, st>>>(
        n, sp, col, val, diag, phi, x1, acc, inv_a, shift, (real)cr[0], (real)ci[0], c1r, c1i);
    TB_CHECK_LAUNCH();
    // t_k alternates between phi's buffer (t_0, t_2, ...) and x1 (t_1, t_3, ...)
    for (int k = 2; k < K; ++k) {
      real *xk = (k & 1) ? phi : x1;   // t_{k-1}
      real *io = (k & 1) ? x1 : phi;   // t_{k-2} in, t_k out
      propagate_term_kernel<real, valT, R, CPT, false><<<grid, kBlock, 0, st>>>(
          n, sp, col, val, diag, xk, io, acc, two_over_a, shift, real(0), real(0), (real)cr[k], (real)ci[k]);
      TB_CHECK_LAUNCH();
    }
    real *t = phi;
    phi = acc;
    acc = t;
    return TB_OK;
  }

  static tb_status run(int64_t n, const int64_t *sp, const int32_t *col, const valT *val, const valT *diag,
                       const valT *vval, double a, double b, int M, uint64_t seed, int64_t r0, int n_steps,
                       double dt, double *mu_out, void *ws, size_t wsb, cudaStream_t st, double *ms_out) {
    const int shape = chosen_shape(sizeof(real) == 4 ? TB_F32 : TB_F64, R, TB_KPM_DIRECT, n);
    if (shape < 0 || shape >= Kit::kShapes) return fail(TB_ERR_INVALID_ARG, "lsqt_vac: step shape %d", shape);
    const int grid = Kit::grid(shape, n, false);
    const int64_t np = padded_rows(n);
    Carver cv(ws, wsb);
    real *vec[kVectors];
    for (int k = 0; k < kVectors; ++k) vec[k] = cv.take<real>((size_t)np * R * 2);
    double *partial = cv.take<double>((size_t)(M + 1) * Kit::max_grid(n) * R);
    int *flags = cv.take<int>(4);
    BandPlan bp;
    BandRec *recs = nullptr;
    uint16_t *lidx = nullptr;
    if (Kit::any_banded()) {
      recs = cv.take<BandRec>(Kit::plan_records(n));
      lidx = cv.take<uint16_t>((size_t)np * kBandSlots);
    }
    if (!cv.ok()) return fail(TB_ERR_WORKSPACE, "lsqt_vac: workspace too small (%zu < %zu)", wsb, cv.used);
    if (Kit::pipelined(shape) && ((reinterpret_cast<uintptr_t>(col) | reinterpret_cast<uintptr_t>(val)) & 15))
      return fail(TB_ERR_INVALID_ARG, "lsqt_vac: col and val must be 16-byte aligned");
    if (Kit::stages_diag(shape) && (reinterpret_cast<uintptr_t>(diag) & 15))
      return fail(TB_ERR_INVALID_ARG, "lsqt_vac: diag must be 16-byte aligned");
    Kit::prepare(shape);
    if (Kit::banded(shape)) {
      bp.recs = recs;
      bp.lidx = lidx;
      const tb_status sp_ = Kit::plan(shape, n, np, sp, col, recs, lidx, st);
      if (sp_ != TB_OK) return sp_;
    }
    real *phi_l = vec[0], *phi_r = vec[1], *w = vec[2], *A = vec[3], *B = vec[4], *x1 = vec[5], *acc = vec[6];
    std::vector<double> cr, ci;
    propagator_coefficients(a, b, dt, cr, ci);
    const real inv_a = static_cast<real>(1.0 / a), two_over_a = static_cast<real>(2.0 / a);
    const real shift = static_cast<real>(b), inv_hbar = static_cast<real>(1.0 / kHbar);
    const int64_t ps = (int64_t)grid * R;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (ms_out) {
      TB_CUDA(cudaEventCreate(&ev[0]));
      TB_CUDA(cudaEventCreate(&ev[1]));
      TB_CUDA(cudaEventRecord(ev[0], st));
    }
    TB_CUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
    lsqt_phase_kernel<real, R><<<(unsigned)((n * R + 255) / 256), 256, 0, st>>>(n, seed, r0, phi_r);
    TB_CHECK_LAUNCH();
    velocity_apply_kernel<real, valT, R, CPT, false><<<grid, kBlock, 0, st>>>(n, sp, col, vval, phi_r, nullptr,
                                                                              phi_l, nullptr, inv_hbar);
    TB_CHECK_LAUNCH();
    BatchTables bt;
    tb_status s = TB_OK;
    for (int j = 0; j <= n_steps && s == TB_OK; ++j) {
      // w = V phi_L and the mu_0 partials Re <w|phi_R>
      velocity_apply_kernel<real, valT, R, CPT, true><<<grid, kBlock, 0, st>>>(n, sp, col, vval, phi_l, phi_r, w,
                                                                               partial, inv_hbar);
      TB_CHECK_LAUNCH();
      // T_m(H~) phi_R, m = 1 .. M-1, dotted with w (A, B alternate; v_2 reads prev = phi_R)
      s = Kit::template step<true, false, false>(shape, grid, n, sp, col, val, diag, phi_r, nullptr, w, A, partial + ps,
                                                 inv_a, shift, flags, ps, bt, st, bp);
      for (int m = 2; m < M && s == TB_OK; ++m) {
        real *out = (m & 1) ? A : B;
        const real *x = (m & 1) ? B : A;
        const real *prev = (m == 2) ? phi_r : out;
        s = Kit::template step<false, false, false>(shape, grid, n, sp, col, val, diag, x, prev, w, out,
                                                    partial + (size_t)m * ps, two_over_a, shift, flags, ps, bt, st,
                                                    bp);
      }
      if (s != TB_OK) break;
      moment_reduce_kernel<<<(M * R + 255) / 256, 256, 0, st>>>(partial, grid, R, M, 1.0 / (double)n, 0, 0.0,
                                                                mu_out + (size_t)j * R * M, flags);
      TB_CHECK_LAUNCH();
      if (j < n_steps) {
        s = propagate(grid, n, sp, col, val, diag, phi_l, x1, acc, inv_a, two_over_a, shift, cr, ci, st);
        if (s == TB_OK)
          s = propagate(grid, n, sp, col, val, diag, phi_r, x1, acc, inv_a, two_over_a, shift, cr, ci, st);
      }
    }
    if (ms_out && s == TB_OK) TB_CUDA(cudaEventRecord(ev[1], st));
    int hflags[4] = {0, 0, 0, 0};
    if (s == TB_OK) {
      TB_CUDA(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
      TB_CUDA(cudaStreamSynchronize(st));
      if (ms_out) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        *ms_out = ms;
      }
    }
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    if (s != TB_OK) return s;
    if (hflags[0] & 4) return fail(TB_ERR_TIMEOUT, "lsqt_vac: a pipeline wait timed out");
    if (hflags[0] & 2) return fail(TB_ERR_NOT_FINITE, "lsqt_vac: non-finite moment");
    return TB_OK;
  }
};

template <typename real, typename valT, int R>
struct LsqtWsOp {
  static tb_status apply(int64_t n, int M, size_t *out) {
    *out = LsqtRunner<real, valT, R>::workspace(n, M);
    return TB_OK;
  }
};

template <typename real, typename valT, int R>
struct LsqtRunOp {
  static tb_status apply(int64_t n, const int64_t *sp, const int32_t *col, const void *val, const void *diag,
                         const void *vval, double a, double b, int M, uint64_t seed, int64_t r0, int n_steps,
                         double dt, double *mu, void *ws, size_t wsb, cudaStream_t st, double *ms) {
    return LsqtRunner<real, valT, R>::run(n, sp, col, static_cast<const valT *>(val),
                                          static_cast<const valT *>(diag), static_cast<const valT *>(vval), a, b,
                                          M, seed, r0, n_steps, dt, mu, ws, wsb, st, ms);
  }
};

template <typename real, typename valT>
struct LsqtDispatch {
  template <template <typename, typename, int> class Op, typename... Args>
  static bool call(int R, tb_status &st, Args... args) {
    switch (R) {
      case 1: st = Op<real, valT, 1>::apply(args...); return true;
      case 2: st = Op<real, valT, 2>::apply(args...); return true;
      case 4: st = Op<real, valT, 4>::apply(args...); return true;
      case 8: st = Op<real, valT, 8>::apply(args...); return true;
      case 16: st = Op<real, valT, 16>::apply(args...); return true;
      default: return false;
    }
  }
};

}  // namespace
}  // namespace gputb

using namespace gputb;

extern "C" tb_status tb_velocity_values(const double *positions, int64_t n, const double *box, const int32_t *pbc,
                                        double rcut, const int64_t *slice_ptr, const int32_t *col, const void *val,
                                        int32_t precision, const double *direction, void *vval, void *stream) {
  TB_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "tb_velocity_values: bad n");
  TB_REQUIRE(positions && slice_ptr && direction && vval, "tb_velocity_values: null pointer argument");
  TB_REQUIRE(precision == TB_F32 || precision == TB_F64, "tb_velocity_values: bad precision");
  TB_REQUIRE(rcut > 0.0, "tb_velocity_values: rcut must be positive");
  Box B;
  tb_status s = make_box(box, pbc, rcut, &B);
  if (s != TB_OK) return s;
  const int64_t n_slices = (n + 31) / 32;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned nb = (unsigned)((n_slices * 32 + 255) / 256);
  if (precision == TB_F32)
    velocity_values_kernel<float><<<nb, 256, 0, st>>>(positions, n, n_slices, B, slice_ptr, col,
                                                      static_cast<const float *>(val), direction[0], direction[1],
                                                      direction[2], static_cast<float *>(vval));
  else
    velocity_values_kernel<double><<<nb, 256, 0, st>>>(positions, n, n_slices, B, slice_ptr, col,
                                                       static_cast<const double *>(val), direction[0], direction[1],
                                                       direction[2], static_cast<double *>(vval));
  TB_CHECK_LAUNCH();
  return TB_OK;
}

extern "C" size_t lsqt_vac_workspace_size(int64_t n, int32_t M, int32_t R, int32_t precision) {
  if (n <= 0 || M < 2) return 0;
  size_t out = 0;
  tb_status st = TB_OK;
  const bool ok = precision == TB_F32 ? LsqtDispatch<float, float>::call<LsqtWsOp>(R, st, n, (int)M, &out)
                                      : LsqtDispatch<double, double>::call<LsqtWsOp>(R, st, n, (int)M, &out);
  return ok ? out : 0;
}

extern "C" tb_status lsqt_vac(int64_t n, const int64_t *slice_ptr, const int32_t *col, const void *val,
                              const void *diag, const void *vval, int32_t precision, double a, double b, int32_t M,
                              int32_t R, uint64_t seed, int64_t first_vector, int32_t n_steps, double dt_fs,
                              double *mu_out, void *workspace, size_t workspace_bytes, void *stream,
                              double *ms_out) {
  TB_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "lsqt_vac: n=%lld out of range", (long long)n);
  TB_REQUIRE(M >= 2, "lsqt_vac: M=%d must be >= 2", M);
  TB_REQUIRE(n_steps >= 0 && n_steps <= 1000000, "lsqt_vac: bad n_steps");
  TB_REQUIRE(dt_fs > 0.0 && std::isfinite(dt_fs), "lsqt_vac: dt must be positive");
  TB_REQUIRE(precision == TB_F32 || precision == TB_F64, "lsqt_vac: bad precision");
  TB_REQUIRE(a > 0.0 && std::isfinite(a) && std::isfinite(b), "lsqt_vac: need finite a > 0, b");
  TB_REQUIRE(a * dt_fs / 0.6582119569 <= 200.0, "lsqt_vac: a*dt/hbar must be <= 200 (shorter time step)");
  TB_REQUIRE(first_vector >= 0 && first_vector <= (int64_t(1) << 31), "lsqt_vac: first_vector out of range");
  TB_REQUIRE(slice_ptr && vval && mu_out && workspace, "lsqt_vac: null pointer argument");
  TB_REQUIRE((reinterpret_cast<uintptr_t>(workspace) & 255) == 0, "lsqt_vac: workspace must be 256-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tb_status status = TB_OK;
  const bool ok =
      precision == TB_F32
          ? LsqtDispatch<float, float>::call<LsqtRunOp>(R, status, n, slice_ptr, col, val, diag, vval, a, b, (int)M,
                                                        seed, first_vector, (int)n_steps, dt_fs, mu_out, workspace,
                                                        workspace_bytes, st, ms_out)
          : LsqtDispatch<double, double>::call<LsqtRunOp>(R, status, n, slice_ptr, col, val, diag, vval, a, b,
                                                          (int)M, seed, first_vector, (int)n_steps, dt_fs, mu_out,
                                                          workspace, workspace_bytes, st, ms_out);
  if (!ok) return fail(TB_ERR_INVALID_ARG, "lsqt_vac: unsupported R=%d", R);
  return status;
}

extern "C" tb_status lsqt_correlation(const double *mu, int32_t n_times, int32_t R, int32_t M, int32_t kernel,
                                      double lambda, double a, double b, const double *energy, int32_t K,
                                      double dt_fs, double *corr, double *sigma, double *coef_ws, void *stream) {
  TB_REQUIRE(n_times >= 1 && R >= 1 && M >= 1 && K >= 1, "lsqt_correlation: bad sizes");
  TB_REQUIRE(mu && energy && corr && coef_ws, "lsqt_correlation: null pointer argument");
  TB_REQUIRE(kernel == TB_KERNEL_JACKSON || kernel == TB_KERNEL_LORENTZ || kernel == TB_KERNEL_NONE,
             "lsqt_correlation: bad kernel");
  TB_REQUIRE(a > 0.0 && dt_fs > 0.0, "lsqt_correlation: need a > 0 and dt > 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t tot = (int64_t)n_times * M;
  vac_coef_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(mu, n_times, R, M, kernel, lambda, coef_ws);
  TB_CHECK_LAUNCH();
  vac_series_kernel<<<(K + 127) / 128, 128, 0, st>>>(coef_ws, n_times, M, a, b, energy, K, dt_fs, corr, sigma);
  TB_CHECK_LAUNCH();
  return TB_OK;
}
