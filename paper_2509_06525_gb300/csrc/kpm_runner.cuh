// KPM moments: random-phase initialisation, the Chebyshev recursion through
// the shared step kernels (kpm_step.cuh), the deterministic moment reduction,
// the batched (segmented, graph-captured) form and the shape autotuner.
// Included once per vector precision (kpm_f32.cu, kpm_f64.cu).
//
// Method (arXiv 2509.06525 Sec. 2.4; conventions of Weisse et al., RMP 78,
// 275 (2006)): H~ = (H - b)/a, v1 = H~ v0, v_{n+1} = 2 H~ v_n - v_{n-1},
// mu_n^(r) = Re <v0_r | v_n_r> / N.
//
// GB300 design
// * The R random vectors form one block-vector stored row-interleaved
//   ([N][R] complex), so each sparse-matrix element that is read from HBM
//   is applied to all R vectors (blocked SpMM; the matrix is read once per
//   step for all vectors).
// * TPR = R / CPT threads share one row; each moves CPT complex numbers with
//   16-byte (or 8-byte) vector accesses, so the gather of a neighbour row is
//   one contiguous, fully used segment.
// * The matrix (col, val) and the row's own v_{n-1}, v0 are streamed
//   (evict-first loads, or bulk copies into a shared-memory ring); the
//   neighbour gathers go through the read-only path and hit L1/L2 because
//   atoms are cell-ordered.
// * v_{n+1} overwrites v_{n-1} in place (each element is read and written by
//   the same thread), so only three vector blocks live in HBM: v0, A, B.
// * The moment partial sums are formed in the same pass (no extra read of
//   v_{n+1}), reduced by warp shuffles and shared memory to one FP64 partial
//   per CTA and step, and summed in a fixed order by a final kernel: results
//   are bitwise reproducible for a given shape.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kpm_entry.h"
#include "kpm_step.cuh"

namespace gputb {
namespace {
using namespace kpmdev;

// v0[i, r] = exp(2 pi i u(seed, r0 + r, i)) (batched: u(seed + s, r, i - row0[s])
// on the real rows of snapshot s, 0 on padding rows); partials of
// Re <v0|v0> per CTA, or per RPB-row block when SEG.
template <typename real, int R, int CPT, bool SEG>
__global__ void __launch_bounds__(kBlock) random_phase_kernel(int64_t n, uint64_t seed, int64_t r0, BatchTables bt,
                                                              real *__restrict__ v0, double *__restrict__ partial) {
  constexpr int TPR = R / CPT;
  constexpr int RPB = kBlock / TPR;
  const int part = threadIdx.x % TPR;
  double acc[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) acc[c] = 0.0;
  for (int64_t row0 = (int64_t)blockIdx.x * RPB; row0 < n; row0 += (int64_t)gridDim.x * RPB) {
    const int64_t i = row0 + threadIdx.x / TPR;
    if (i < n) {
      uint64_t sd = seed;
      int64_t li = i;
      bool real_row = true;
      if (bt.tile_snap) {
        const int s = bt.tile_snap[i / kBatchTile];
        sd = seed + (uint64_t)s;
        li = i - bt.row0[s];
        real_row = li < bt.rows[s];
      }
      real v[2 * CPT];
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int r = part * CPT + c;
        real sn = real(0), co = real(0);
        if (real_row) phase_cis<real>(sd, (uint64_t)(r0 + r), (uint64_t)li, co, sn);
        v[2 * c] = co;
        v[2 * c + 1] = sn;
        acc[c] += (double)v[2 * c] * (double)v[2 * c] + (double)v[2 * c + 1] * (double)v[2 * c + 1];
      }
      st_stream<real, CPT>(v0 + (i * R + part * CPT) * 2, v);
    }
    if (SEG) {
      cta_partial<R, CPT>(acc, partial + (row0 / RPB) * R);
      __syncthreads();
#pragma unroll
      for (int c = 0; c < CPT; ++c) acc[c] = 0.0;
    }
  }
  if (!SEG) cta_partial<R, CPT>(acc, partial + (int64_t)blockIdx.x * R);
}

// batched reduction, step 1: one warp per (snapshot s, moment slot m) sums
// the slot's block partials of s -- a contiguous run of (b1 - b0) R doubles,
// read coalesced; lane l takes entries l, l + 32, ... (vector l mod R), then
// lanes of one vector are added in a fixed shuffle tree -- and writes the
// raw sums S_m into mu[s][r][m] (deterministic)
__global__ void batched_slot_sum_kernel(BatchTables bt, int M, int R, int rpb, int64_t nblk,
                                        const double *__restrict__ partial, double *__restrict__ mu) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (int64_t)bt.n_snap * M) return;
  const int s = static_cast<int>(w / M), m = static_cast<int>(w % M);
  const int64_t rows = bt.rows[s];
  const int64_t b0 = bt.row0[s] / rpb;
  const int64_t b1 = (bt.row0[s] + (rows + kBatchTile - 1) / kBatchTile * kBatchTile) / rpb;
  const double *p = partial + (int64_t)m * nblk * R + b0 * R;
  const int64_t cnt = (b1 - b0) * R;
  double acc = 0.0;
  for (int64_t e = lane; e < cnt; e += 32) acc += p[e];
  for (int off = 16; off >= R; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane < R) mu[((int64_t)s * R + lane) * M + m] = acc;
}

// step 2: one thread per (snapshot, vector) turns the raw sums into moments
// in place: mu_m = S_m / n, and in doubling mode mu_m = 2 S_m / n - mu_(m mod 2)
// for m >= 2 (Weisse et al. 2006)
__global__ void batched_moments_kernel(BatchTables bt, int M, int R, int doubling, double *__restrict__ mu,
                                       int *__restrict__ flags) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)bt.n_snap * R) return;
  const int s = static_cast<int>(t / R);
  double *row = mu + t * M;
  const double inv_n = 1.0 / (double)bt.rows[s];
  const double mu0 = row[0] * inv_n, mu1 = M > 1 ? row[1] * inv_n : 0.0;
  bool bad = false, big = false;
  for (int m = 0; m < M; ++m) {
    double v = m == 0 ? mu0 : (m == 1 ? mu1 : row[m] * inv_n);
    if (doubling && m >= 2) v = 2.0 * v - ((m & 1) ? mu1 : mu0);
    row[m] = v;
    bad = bad || !isfinite(v);
    big = big || fabs(v) > 1.0 + 1e-6;
  }
  if (bad) atomicOr(flags, 2);
  else if (big) atomicOr(flags, 1);
}

template <typename real, typename valT, int R>
struct KpmRunner {
  using Kit = StepKit<real, valT, R>;
  static constexpr int64_t kRowPad = Kit::kRowPad;

  static int64_t padded_rows(int64_t n) { return (n + kRowPad - 1) / kRowPad * kRowPad; }

  // band plan storage (banded shapes only): records, then local indices
  struct PlanWs {
    BandRec *recs = nullptr;
    uint16_t *lidx = nullptr;
  };
  static void carve_plan(Carver &cv, int64_t n, PlanWs *pw) {
    if (!Kit::any_banded()) return;
    pw->recs = cv.take<BandRec>(Kit::plan_records(n));
    pw->lidx = cv.take<uint16_t>((size_t)padded_rows(n) * kBandSlots);
  }

  static size_t workspace(int64_t n, int M, bool segmented) {
    Carver cv(nullptr, 0);
    for (int k = 0; k < 3; ++k) cv.take<real>((size_t)padded_rows(n) * R * 2);
    const int64_t units = segmented ? (n + Kit::min_rows_per_block() - 1) / Kit::min_rows_per_block()
                                    : Kit::max_grid(n);
    cv.take<double>((size_t)(M + 1) * units * R);
    cv.take<int>(4);
    PlanWs pw;
    carve_plan(cv, n, &pw);
    return cv.used + 256;
  }

  // the band plan of `shape` (a no-op for shapes that need none)
  static tb_status make_plan(int shape, int64_t n, const int64_t *slice_ptr, const int32_t *col, const PlanWs &pw,
                             cudaStream_t st, BandPlan *bp) {
    if (!Kit::banded(shape)) return TB_OK;
    bp->recs = pw.recs;
    bp->lidx = pw.lidx;
    return Kit::plan(shape, n, padded_rows(n), slice_ptr, col, pw.recs, pw.lidx, st);
  }

  static tb_status random_phases(int shape, int grid, int64_t n, uint64_t seed, int64_t r0, const BatchTables &bt,
                                 bool seg, real *v0, double *partial, cudaStream_t st) {
    return visit_shape<real, valT, R>(shape, [&](auto k) {
      constexpr int C = R / decltype(k)::TPR;
      if (seg)
        random_phase_kernel<real, R, C, true><<<grid, kBlock, 0, st>>>(n, seed, r0, bt, v0, partial);
      else
        random_phase_kernel<real, R, C, false><<<grid, kBlock, 0, st>>>(n, seed, r0, bt, v0, partial);
      TB_CHECK_LAUNCH();
      return TB_OK;
    });
  }

  // The whole recursion: random phases, the Chebyshev steps, the reduction.
  template <bool SEG>
  static tb_status enqueue(int shape, int grid, int64_t n, const int64_t *slice_ptr, const int32_t *col,
                           const valT *val, const valT *diag, double a, double b, int M, uint64_t seed, int64_t r0,
                           bool dbl, double *mu_r, real *v0, real *A, real *B, double *partial, int *flags,
                           const BatchTables &bt, cudaStream_t st, cudaEvent_t ev_begin, cudaEvent_t ev_end,
                           const BandPlan &bp) {
    const int rpb = Kit::rows_per_block(shape);
    const int64_t units = SEG ? (n + rpb - 1) / rpb : grid;   // partials per moment slot
    const int64_t ps = units * R;
    TB_CUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
    tb_status s = random_phases(shape, grid, n, seed, r0, bt, SEG, v0, partial, st);
    if (s != TB_OK) return s;
    if (ev_begin) TB_CUDA(cudaEventRecord(ev_begin, st));
    // v1 = H~ v0 -> A.  Direct mode: the step making v_m adds the partials of
    // mu_m; doubling mode: the step reading v_k adds those of S_2k and S_2k+1.
    const real shift = static_cast<real>(b);
    const real inv_a = static_cast<real>(1.0 / a);
    s = dbl ? Kit::template step<true, true, SEG>(shape, grid, n, slice_ptr, col, val, diag, v0, nullptr, v0, A,
                                                  partial, inv_a, shift, flags, ps, bt, st, bp)
            : Kit::template step<true, false, SEG>(shape, grid, n, slice_ptr, col, val, diag, v0, nullptr, v0, A,
                                                   partial + ps, inv_a, shift, flags, ps, bt, st, bp);
    if (s != TB_OK) return s;
    const real two_over_a = static_cast<real>(2.0 / a);
    const int last = dbl ? (M - 1) / 2 + 1 : M - 1;   // index of the last vector computed
    for (int m = 2; m <= last; ++m) {
      // v_m is written over v_{m-2}: m even -> B, m odd -> A; v_2 reads prev = v0
      real *out = (m & 1) ? A : B;
      const real *x = (m & 1) ? B : A;
      const real *prev = (m == 2) ? v0 : out;
      s = dbl ? Kit::template step<false, true, SEG>(shape, grid, n, slice_ptr, col, val, diag, x, prev, v0, out,
                                                     partial + (size_t)(2 * (m - 1)) * ps, two_over_a, shift,
                                                     flags, ps, bt, st, bp)
              : Kit::template step<false, false, SEG>(shape, grid, n, slice_ptr, col, val, diag, x, prev, v0, out,
                                                      partial + (size_t)m * ps, two_over_a, shift, flags, ps, bt,
                                                      st, bp);
      if (s != TB_OK) return s;
    }
    if (ev_end) TB_CUDA(cudaEventRecord(ev_end, st));
    if (SEG) {
      const int64_t warps = (int64_t)bt.n_snap * M;
      batched_slot_sum_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(bt, M, R, rpb, units, partial,
                                                                                     mu_r);
      TB_CHECK_LAUNCH();
      const int64_t vecs = (int64_t)bt.n_snap * R;
      batched_moments_kernel<<<(unsigned)((vecs + 127) / 128), 128, 0, st>>>(bt, M, R, dbl ? 1 : 0, mu_r, flags);
    } else {
      const int total = M * R;
      moment_reduce_kernel<<<(total + 255) / 256, 256, 0, st>>>(partial, grid, R, M, 1.0 / (double)n, dbl ? 1 : 0,
                                                                1.0 + 1e-6, mu_r, flags);
    }
    TB_CHECK_LAUNCH();
    return TB_OK;
  }

  static tb_status check_flags(const int *flags, cudaStream_t st, const char *who) {
    int hflags[4] = {0, 0, 0, 0};
    TB_CUDA(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
    TB_CUDA(cudaStreamSynchronize(st));
    if (hflags[0] & 4) return fail(TB_ERR_TIMEOUT, "%s: a pipeline wait timed out", who);
    if (hflags[0] & 2) return fail(TB_ERR_NOT_FINITE, "%s: non-finite moment", who);
    if (hflags[0] & 1)
      return fail(TB_ERR_BOUNDS, "%s: |mu_n| > 1 + 1e-6; the spectrum is not inside [b - a, b + a]", who);
    return TB_OK;
  }

  static tb_status check_alignment(int shape, const int32_t *col, const valT *val, const valT *diag,
                                   const char *who) {
    if (Kit::pipelined(shape) && ((reinterpret_cast<uintptr_t>(col) | reinterpret_cast<uintptr_t>(val)) & 15))
      return fail(TB_ERR_INVALID_ARG, "%s: col and val must be 16-byte aligned", who);
    if (Kit::stages_diag(shape) && (reinterpret_cast<uintptr_t>(diag) & 15))
      return fail(TB_ERR_INVALID_ARG, "%s: diag must be 16-byte aligned", who);
    return TB_OK;
  }

  static tb_status run(int shape, int64_t n, const int64_t *slice_ptr, const int32_t *col, const valT *val,
                       const valT *diag, double a, double b, int M, uint64_t seed, int64_t r0, int mode,
                       double *mu_r, void *ws, size_t ws_bytes, cudaStream_t st, double *step_ms) {
    const bool dbl = mode == TB_KPM_DOUBLING;
    const int grid = Kit::grid(shape, n, dbl);
    const int64_t np = padded_rows(n);
    Carver cv(ws, ws_bytes);
    real *v0 = cv.take<real>((size_t)np * R * 2);
    real *A = cv.take<real>((size_t)np * R * 2);
    real *B = cv.take<real>((size_t)np * R * 2);
    double *partial = cv.take<double>((size_t)(M + 1) * Kit::max_grid(n) * R);
    int *flags = cv.take<int>(4);
    PlanWs pw;
    carve_plan(cv, n, &pw);
    if (!cv.ok()) return fail(TB_ERR_WORKSPACE, "kpm_moments: workspace too small (%zu < %zu)", ws_bytes, cv.used);
    tb_status s = check_alignment(shape, col, val, diag, "kpm_moments");
    if (s != TB_OK) return s;
    Kit::prepare(shape);
    BandPlan bp;
    s = make_plan(shape, n, slice_ptr, col, pw, st, &bp);
    if (s != TB_OK) return s;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (step_ms) {
      TB_CUDA(cudaEventCreate(&ev[0]));
      TB_CUDA(cudaEventCreate(&ev[1]));
    }
    s = enqueue<false>(shape, grid, n, slice_ptr, col, val, diag, a, b, M, seed, r0, dbl, mu_r, v0, A, B, partial,
                       flags, BatchTables(), st, ev[0], ev[1], bp);
    if (s == TB_OK) s = check_flags(flags, st, "kpm_moments");
    if (step_ms) {
      float ms = 0.f;
      if (s == TB_OK) cudaEventElapsedTime(&ms, ev[0], ev[1]);
      *step_ms = ms;
      cudaEventDestroy(ev[0]);
      cudaEventDestroy(ev[1]);
    }
    return s;
  }

  // Batched: the caller's block-diagonal, already rescaled matrix of n_pad
  // rows (see kpm_moments_batched).  Enqueues the band plan (banded shapes),
  // the random phases, the recursion and the segmented reduction on `st`
  // (which kpm_moments_batched captures into a CUDA graph); *flags_out
  // receives the status flags to check after the launch.
  static tb_status enqueue_batched(int shape, int64_t n_pad, const int64_t *slice_ptr, const int32_t *col,
                                   const valT *val, const valT *diag, int M, uint64_t seed, int mode,
                                   const BatchTables &bt, double *mu, void *ws, size_t ws_bytes, cudaStream_t st,
                                   int **flags_out) {
    const bool dbl = mode == TB_KPM_DOUBLING;
    const int grid = Kit::grid(shape, n_pad, dbl);
    Carver cv(ws, ws_bytes);
    real *v0 = cv.take<real>((size_t)n_pad * R * 2);
    real *A = cv.take<real>((size_t)n_pad * R * 2);
    real *B = cv.take<real>((size_t)n_pad * R * 2);
    double *partial = cv.take<double>((size_t)(M + 1) * ((n_pad + Kit::min_rows_per_block() - 1) /
                                                         Kit::min_rows_per_block()) * R);
    int *flags = cv.take<int>(4);
    PlanWs pw;
    carve_plan(cv, n_pad, &pw);
    if (!cv.ok()) return fail(TB_ERR_WORKSPACE, "kpm_moments_batched: workspace too small");
    *flags_out = flags;
    BandPlan bp;
    tb_status s = make_plan(shape, n_pad, slice_ptr, col, pw, st, &bp);
    if (s != TB_OK) return s;
    return enqueue<true>(shape, grid, n_pad, slice_ptr, col, val, diag, 1.0, 0.0, M, seed, 0, dbl, mu, v0, A, B,
                         partial, flags, bt, st, nullptr, nullptr, bp);
  }

  // Autotuner: v0 from the random phases, v1 = H~ v0 with the default shape,
  // then for every candidate shape two warm-up steps and `reps` timed steps of
  // the recursion (the same kernels, operands and in-place update as a
  // kpm_moments call; CUDA events on `st`).  SEG: the segmented step of a
  // block-diagonal batch (tables bt), as kpm_moments_batched runs it.
  template <bool SEG>
  static tb_status autotune(int64_t n, const int64_t *slice_ptr, const int32_t *col, const valT *val,
                            const valT *diag, double a, double b, int mode, int reps, void *ws, size_t ws_bytes,
                            cudaStream_t st, int *best, float *ms_out, int ms_capacity, const BatchTables &bt) {
    const bool dbl = mode == TB_KPM_DOUBLING;
    const int64_t np = padded_rows(n);
    // partial slots per moment: one per CTA, or (segmented) one per row block
    auto units = [&](int shape) -> int64_t {
      return SEG ? (n + Kit::rows_per_block(shape) - 1) / Kit::rows_per_block(shape) : (int64_t)Kit::max_grid(n);
    };
    const int64_t umax = SEG ? (n + Kit::min_rows_per_block() - 1) / Kit::min_rows_per_block() : units(0);
    Carver cv(ws, ws_bytes);
    real *v0 = cv.take<real>((size_t)np * R * 2);
    real *A = cv.take<real>((size_t)np * R * 2);
    real *B = cv.take<real>((size_t)np * R * 2);
    double *partial = cv.take<double>((size_t)3 * umax * R);
    int *flags = cv.take<int>(4);
    PlanWs pw;
    carve_plan(cv, n, &pw);
    if (!cv.ok()) return fail(TB_ERR_WORKSPACE, "tb_kpm_autotune: workspace too small (%zu < %zu)", ws_bytes, cv.used);
    const real shift = static_cast<real>(b);
    const real inv_a = static_cast<real>(1.0 / a), two_over_a = static_cast<real>(2.0 / a);
    TB_CUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
    tb_status s = random_phases(0, Kit::grid(0, n, dbl), n, 42, 0, bt, SEG, v0, partial, st);
    if (s != TB_OK) return s;
    for (int shape = 0; shape < Kit::kShapes; ++shape) {
      s = check_alignment(shape, col, val, diag, "tb_kpm_autotune");
      if (s != TB_OK) return s;
    }
    Kit::prepare(0);
    s = Kit::template step<true, false, SEG>(0, Kit::grid(0, n, false), n, slice_ptr, col, val, diag, v0, nullptr,
                                             v0, A, partial, inv_a, shift, flags, units(0) * R, bt, st);
    if (s != TB_OK) return s;
    TB_CUDA(cudaMemcpyAsync(B, v0, (size_t)np * R * 2 * sizeof(real), cudaMemcpyDeviceToDevice, st));
    cudaEvent_t ev[2];
    TB_CUDA(cudaEventCreate(&ev[0]));
    TB_CUDA(cudaEventCreate(&ev[1]));
    float best_ms = 0.f;
    *best = 0;
    for (int shape = 0; shape < Kit::kShapes && s == TB_OK; ++shape) {
      Kit::prepare(shape);
      const int grid = Kit::grid(shape, n, dbl);
      BandPlan bp;
      s = make_plan(shape, n, slice_ptr, col, pw, st, &bp);
      if (s != TB_OK) break;
      const int64_t ps = units(shape) * R;
      auto one = [&](int k) {
        // the recursion's in-place update: out = 2 H~ x - out
        real *out = (k & 1) ? A : B;
        const real *x = (k & 1) ? B : A;
        return dbl ? Kit::template step<false, true, SEG>(shape, grid, n, slice_ptr, col, val, diag, x, out, v0,
                                                          out, partial, two_over_a, shift, flags, ps, bt, st, bp)
                   : Kit::template step<false, false, SEG>(shape, grid, n, slice_ptr, col, val, diag, x, out, v0,
                                                           out, partial, two_over_a, shift, flags, ps, bt, st, bp);
      };
      for (int k = 0; k < 2 && s == TB_OK; ++k) s = one(k);
      if (s != TB_OK) break;
      if (cudaEventRecord(ev[0], st) != cudaSuccess) s = fail(TB_ERR_CUDA, "tb_kpm_autotune: event record");
      for (int k = 0; k < reps && s == TB_OK; ++k) s = one(k);
      if (s != TB_OK) break;
      float ms = 0.f;
      if (cudaEventRecord(ev[1], st) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess ||
          cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) {
        s = fail(TB_ERR_CUDA, "tb_kpm_autotune: event timing failed");
        break;
      }
      ms /= (float)reps;
      if (ms_out && shape < ms_capacity) ms_out[shape] = ms;
      if (shape == 0 || ms < best_ms) {
        best_ms = ms;
        *best = shape;
      }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (s != TB_OK) return s;
    int hflags[4] = {0, 0, 0, 0};
    TB_CUDA(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
    TB_CUDA(cudaStreamSynchronize(st));
    if (hflags[0] & 4) return fail(TB_ERR_TIMEOUT, "tb_kpm_autotune: a pipeline wait timed out");
    return TB_OK;
  }
};

// Calls Op<real, valT, R>::apply(args...) for the runtime R; false if R is
// not supported.
template <typename real, typename valT>
struct KpmDispatch {
  template <template <typename, typename, int> class Op, typename... Args>
  static bool call(int R, Args &&...args) {
    switch (R) {
      case 1: Op<real, valT, 1>::apply(std::forward<Args>(args)...); return true;
      case 2: Op<real, valT, 2>::apply(std::forward<Args>(args)...); return true;
      case 4: Op<real, valT, 4>::apply(std::forward<Args>(args)...); return true;
      case 8: Op<real, valT, 8>::apply(std::forward<Args>(args)...); return true;
      case 16: Op<real, valT, 16>::apply(std::forward<Args>(args)...); return true;
      case 32: Op<real, valT, 32>::apply(std::forward<Args>(args)...); return true;
      default: return false;
    }
  }
};

template <typename real, typename valT, int R>
struct CountOp {
  static void apply(int *out) { *out = StepKit<real, valT, R>::kShapes; }
};
template <typename real, typename valT, int R>
struct InfoOp {
  static void apply(int shape, tb_step_shape *out, bool *ok) {
    using Kit = StepKit<real, valT, R>;
    *ok = shape >= 0 && shape < Kit::kShapes;
    if (!*ok) return;
    const StepShape &sh = Shapes<real, R>::at[shape];
    out->pipelined = sh.kind;
    out->complex_per_thread = sh.cpt;
    out->stages = sh.kind ? sh.stages : 0;
    out->min_blocks = sh.minb;
    out->rows_per_tile = Kit::rows_per_block(shape);
    out->rows_per_thread = sh.kind == 2 ? sh.rpt : 1;
    out->staged_vectors = sh.kind == 0 ? 0 : sh.svec;
    out->options = sh.opt;
    out->band_rows = sh.kind == 3 ? sh.brows : 0;
  }
};
template <typename real, typename valT, int R>
struct GridOp {
  static void apply(int shape, int64_t n, bool dbl, int *out) {
    using Kit = StepKit<real, valT, R>;
    *out = (shape >= 0 && shape < Kit::kShapes) ? Kit::grid(shape, n, dbl) : -1;
  }
};
template <typename real, typename valT, int R>
struct WsOp {
  static void apply(int64_t n, int M, bool seg, size_t *out) { *out = KpmRunner<real, valT, R>::workspace(n, M, seg); }
};
template <typename real, typename valT, int R>
struct RunOp {
  static void apply(tb_status *status, int shape, int64_t n, const int64_t *sp, const int32_t *col, const void *val,
                    const void *diag, double a, double b, int M, uint64_t seed, int64_t r0, int mode, double *mu,
                    void *ws, size_t wsb, cudaStream_t st, double *step_ms) {
    if (shape < 0 || shape >= StepKit<real, valT, R>::kShapes) {
      *status = fail(TB_ERR_INVALID_ARG, "kpm_moments: step shape %d out of range", shape);
      return;
    }
    *status = KpmRunner<real, valT, R>::run(shape, n, sp, col, static_cast<const valT *>(val),
                                            static_cast<const valT *>(diag), a, b, M, seed, r0, mode, mu, ws, wsb,
                                            st, step_ms);
  }
};
template <typename real, typename valT, int R>
struct PrepOp {
  static void apply(int shape, bool *ok) {
    using Kit = StepKit<real, valT, R>;
    *ok = shape >= 0 && shape < Kit::kShapes;
    if (*ok) Kit::prepare(shape);
  }
};
template <typename real, typename valT, int R>
struct BatchEnqueueOp {
  static void apply(tb_status *status, int shape, int64_t n_pad, const int64_t *sp, const int32_t *col,
                    const void *val, const void *diag, int M, uint64_t seed, int mode, const BatchDesc &bd,
                    double *mu, void *ws, size_t wsb, cudaStream_t st, int **flags) {
    if (shape < 0 || shape >= StepKit<real, valT, R>::kShapes) {
      *status = fail(TB_ERR_INVALID_ARG, "kpm_moments_batched: step shape %d out of range", shape);
      return;
    }
    BatchTables bt;
    bt.tile_snap = bd.tile_snap;
    bt.row0 = bd.row0;
    bt.rows = bd.rows;
    bt.n_snap = bd.n_snap;
    *status = KpmRunner<real, valT, R>::enqueue_batched(shape, n_pad, sp, col, static_cast<const valT *>(val),
                                                        static_cast<const valT *>(diag), M, seed, mode, bt, mu, ws,
                                                        wsb, st, flags);
  }
};
template <typename real, typename valT, int R>
struct TuneOp {
  static void apply(tb_status *status, int64_t n, const int64_t *sp, const int32_t *col, const void *val,
                    const void *diag, double a, double b, int mode, int reps, void *ws, size_t wsb, cudaStream_t st,
                    int *best, float *ms, int cap, const BatchDesc *bd) {
    using Run = KpmRunner<real, valT, R>;
    if (bd) {
      BatchTables bt;
      bt.tile_snap = bd->tile_snap;
      bt.row0 = bd->row0;
      bt.rows = bd->rows;
      bt.n_snap = bd->n_snap;
      *status = Run::template autotune<true>(n, sp, col, static_cast<const valT *>(val),
                                             static_cast<const valT *>(diag), a, b, mode, reps, ws, wsb, st, best, ms,
                                             cap, bt);
    } else {
      *status = Run::template autotune<false>(n, sp, col, static_cast<const valT *>(val),
                                              static_cast<const valT *>(diag), a, b, mode, reps, ws, wsb, st, best,
                                              ms, cap, BatchTables());
    }
  }
};

}  // namespace
}  // namespace gputb

// Defines KpmEntry<real> for one vector precision (values of the same type).
#define GPUTB_DEFINE_KPM_ENTRY(REAL)                                                                               \
  namespace gputb {                                                                                                \
  namespace kpmdev {                                                                                               \
  template <>                                                                                                      \
  bool KpmEntry<REAL>::shape_count(int R, int *count) {                                                            \
    return KpmDispatch<REAL, REAL>::call<CountOp>(R, count);                                                       \
  }                                                                                                                \
  template <>                                                                                                      \
  bool KpmEntry<REAL>::shape_info(int R, int shape, tb_step_shape *out) {                                          \
    bool ok = false;                                                                                               \
    return KpmDispatch<REAL, REAL>::call<InfoOp>(R, shape, out, &ok) && ok;                                        \
  }                                                                                                                \
  template <>                                                                                                      \
  bool KpmEntry<REAL>::shape_grid(int R, int shape, int64_t n, bool doubling, int *out) {                          \
    return KpmDispatch<REAL, REAL>::call<GridOp>(R, shape, n, doubling, out);                                      \
  }                                                                                                                \
  template <>                                                                                                      \
  bool KpmEntry<REAL>::workspace(int R, int64_t n, int M, bool segmented, size_t *out) {                           \
    return KpmDispatch<REAL, REAL>::call<WsOp>(R, n, M, segmented, out);                                           \
  }                                                                                                                \
  template <>                                                                                                      \
  bool KpmEntry<REAL>::run(int R, tb_status *status, int shape, int64_t n, const int64_t *slice_ptr,              \
                           const int32_t *col, const void *val, const void *diag, double a, double b, int M,      \
                           uint64_t seed, int64_t r0, int mode, double *mu_r, void *ws, size_t ws_bytes,          \
                           cudaStream_t st, double *step_ms) {                                                    \
    return KpmDispatch<REAL, REAL>::call<RunOp>(R, status, shape, n, slice_ptr, col, val, diag, a, b, M, seed,    \
                                                r0, mode, mu_r, ws, ws_bytes, st, step_ms);                       \
  }                                                                                                                \
  template <>                                                                                                      \
  bool KpmEntry<REAL>::prepare(int R, int shape) {                                                                 \
    bool ok = false;                                                                                               \
    return KpmDispatch<REAL, REAL>::call<PrepOp>(R, shape, &ok) && ok;                                             \
  }                                                                                                                \
  template <>                                                                                                      \
  bool KpmEntry<REAL>::enqueue_batched(int R, tb_status *status, int shape, int64_t n_pad,                         \
                                       const int64_t *slice_ptr, const int32_t *col, const void *val,              \
                                       const void *diag, int M, uint64_t seed, int mode, const BatchDesc &bt,      \
                                       double *mu, void *ws, size_t ws_bytes, cudaStream_t st, int **flags) {      \
    return KpmDispatch<REAL, REAL>::call<BatchEnqueueOp>(R, status, shape, n_pad, slice_ptr, col, val, diag, M,   \
                                                         seed, mode, bt, mu, ws, ws_bytes, st, flags);             \
  }                                                                                                                \
  template <>                                                                                                      \
  bool KpmEntry<REAL>::autotune(int R, tb_status *status, int64_t n, const int64_t *slice_ptr, const int32_t *col, \
                                const void *val, const void *diag, double a, double b, int mode, int reps,         \
                                void *ws, size_t ws_bytes, cudaStream_t st, int *best, float *ms,                  \
                                int ms_capacity, const BatchDesc *bt) {                                            \
    return KpmDispatch<REAL, REAL>::call<TuneOp>(R, status, n, slice_ptr, col, val, diag, a, b, mode, reps, ws,   \
                                                 ws_bytes, st, best, ms, ms_capacity, bt);                         \
  }                                                                                                                \
  }                                                                                                                \
  }
