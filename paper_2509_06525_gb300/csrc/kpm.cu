// KPM moments: random-phase initialisation, the Chebyshev step fused with
// the moment dot products, and the deterministic moment reduction.
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
//   one 16-byte (or 8-byte for R = 1 in FP32) vector access, so the gather of
//   a neighbour row is one contiguous, fully used segment.
// * The matrix (col, val) and the row's own v_{n-1}, v0 are streamed with
//   evict-first loads; the neighbour gathers go through the read-only path
//   and hit L1/L2 because atoms are cell-ordered.
// * v_{n+1} overwrites v_{n-1} in place (each element is read and written by
//   the same thread), so only three vector blocks live in HBM: v0, A, B.
// * The moment partial sums Re(conj(v0) v_{n+1}) are formed in the same pass
//   (no extra read of v_{n+1}), accumulated in FP64, reduced by warp
//   shuffles and shared memory to one partial per CTA and step, and summed
//   in a fixed order by a final kernel: results are bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kpm_step.cuh"
#include "kpm_fused.cuh"

namespace gputb {
namespace kpmdev {
int g_kpm_variant = 0;
}  // namespace kpmdev
namespace {
using namespace kpmdev;

constexpr int kMaxPairGrid = 4096;   // CTAs of a cooperative pair launch (at most)

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

// batched: mu[s][r][m] from the RPB-row block partials of snapshot s (block order)
__global__ void batched_reduce_kernel(BatchTables bt, int M, int R, int rpb, int64_t nblk,
                                      const double *__restrict__ partial, int doubling, double *__restrict__ mu,
                                      int *__restrict__ flags) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)bt.n_snap * R * M) return;
  const int m = static_cast<int>(t % M);
  const int r = static_cast<int>((t / M) % R);
  const int s = static_cast<int>(t / ((int64_t)M * R));
  const int64_t rows = bt.rows[s];
  const int64_t b0 = bt.row0[s] / rpb;
  const int64_t b1 = (bt.row0[s] + (rows + kBatchTile - 1) / kBatchTile * kBatchTile) / rpb;
  const double inv_n = 1.0 / (double)rows;
  auto slot = [&](int k) {
    const double *p = partial + (int64_t)k * nblk * R + r;
    double acc = 0.0;
    for (int64_t q = b0; q < b1; ++q) acc += p[q * R];
    return acc * inv_n;
  };
  double v = slot(m);
  if (doubling && m >= 2) v = 2.0 * v - slot(m & 1);
  mu[t] = v;
  if (!isfinite(v)) atomicOr(flags, 2);
  else if (fabs(v) > 1.0 + 1e-6) atomicOr(flags, 1);
}

template <typename real, typename valT, int R>
struct KpmRunner : StepKit<real, valT, R> {
  using Kit = StepKit<real, valT, R>;
  using Kit::CPT;
  using Kit::TPR;
  using Kit::RPB;
  using typename Kit::G;
  using Kit::use_bulk;
  using Kit::grid_for;
  using Kit::prepare;
  static constexpr int64_t kRowPad = Kit::kRowPad;

  static int64_t padded_rows(int64_t n) { return (n + kRowPad - 1) / kRowPad * kRowPad; }
  static int64_t blocks(int64_t n) { return (n + RPB - 1) / RPB; }   // RPB == G::TR

  static size_t workspace(int64_t n, int M, bool segmented) {
    Carver cv(nullptr, 0);
    for (int k = 0; k < 3; ++k) cv.take<real>((size_t)padded_rows(n) * R * 2);
    const int64_t units = segmented ? blocks(n) : std::max(grid_for(n, false), grid_for(n, true));
    cv.take<double>((size_t)(M + 1) * units * R);
    cv.take<int>(4);
    if (!segmented) {
      PairWs pw;
      carve_pair(cv, n, M, &pw);
    }
    return cv.used + 256;
  }

  // ---- two steps per launch (kpm_fused.cuh) ----
  struct PairWs {
    PairPlan plan;
    int32_t *tasks;
    int2 *wait;
    int *lo, *hi, *rlo, *rhi, *key, *fill;
    int64_t *gsize, *gtotal;
    void *scan_ws;
    double *bpart;
  };

  static void carve_pair(Carver &cv, int64_t n, int M, PairWs *w) {
    (void)M;
    const int64_t nb = blocks(n);
    w->tasks = cv.take<int32_t>(2 * nb);
    w->wait = cv.take<int2>(nb);
    w->plan.done = cv.take<int>(nb);
    w->plan.cta_s1 = cv.take<int>(kMaxPairGrid);
    w->lo = cv.take<int>(nb);
    w->hi = cv.take<int>(nb);
    w->rlo = cv.take<int>(nb);
    w->rhi = cv.take<int>(nb);
    w->key = cv.take<int>(nb);
    w->fill = cv.take<int>(nb);
    w->gsize = cv.take<int64_t>(nb + 1);
    w->gtotal = cv.take<int64_t>(1);
    w->scan_ws = cv.take<char>(scan_workspace_bytes(nb + 1));
    w->bpart = cv.take<double>((size_t)4 * nb * R);
    w->plan.tasks = w->tasks;
    w->plan.wait = w->wait;
    w->plan.nb = nb;
  }

  // opt-in only: on GB300 the per-task latency chain (task, slice offsets,
  // columns, gathers) with one row per thread costs more than the L2 reuse
  // saves (measured 2.1x slower than single steps at 1e8 atoms, R = 1)
  static bool use_pair(bool dbl) { return dbl && g_kpm_variant == 3; }

  // resident CTAs of the cooperative pair launch
  static int pair_grid() {
    static int per_sm = 0;
    if (per_sm == 0) {
      int b = 0;
      cudaError_t e;
      if (use_bulk()) {
        using GP = BulkGeom<real, valT, R, CPT, 1>;
        cudaFuncSetAttribute(cheb_pair_bulk_kernel<real, valT, R, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)GP::kSmem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cheb_pair_bulk_kernel<real, valT, R, CPT>, kBlock,
                                                          GP::kSmem);
      } else {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cheb_pair_kernel<real, valT, R, CPT>, kBlock, 0);
      }
      per_sm = (e != cudaSuccess || b <= 0) ? 1 : b;
    }
    const int g = per_sm * sm_count();
    return g < kMaxPairGrid ? g : kMaxPairGrid;
  }

  // the task list of the matrix (see kpm_fused.cuh); lag = the grid size
  static tb_status build_pair_plan(int64_t n, const int64_t *slice_ptr, const int32_t *col, PairWs &w,
                                   cudaStream_t st) {
    const int64_t nb = w.plan.nb;
    TB_CUDA(cudaMemsetAsync(w.plan.done, 0, nb * sizeof(int), st));
    TB_CUDA(cudaMemsetAsync(w.plan.cta_s1, 0, kMaxPairGrid * sizeof(int), st));
    TB_CUDA(cudaMemsetAsync(w.lo, 0x7f, nb * sizeof(int), st));
    TB_CUDA(cudaMemsetAsync(w.hi, 0xff, nb * sizeof(int), st));
    TB_CUDA(cudaMemsetAsync(w.rlo, 0x7f, nb * sizeof(int), st));
    TB_CUDA(cudaMemsetAsync(w.rhi, 0xff, nb * sizeof(int), st));
    TB_CUDA(cudaMemsetAsync(w.fill, 0, nb * sizeof(int), st));
    pair_hull_kernel<RPB><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, slice_ptr, col, w.lo, w.hi, w.rlo, w.rhi);
    TB_CHECK_LAUNCH();
    fill_ones_kernel<<<(unsigned)((nb + 1 + 255) / 256), 256, 0, st>>>(nb + 1, w.gsize);
    TB_CHECK_LAUNCH();
    pair_wait_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(
        nb, pair_grid(), w.lo, w.hi, w.rlo, w.rhi, w.wait, w.key, reinterpret_cast<unsigned long long *>(w.gsize));
    TB_CHECK_LAUNCH();
    tb_status s = exclusive_scan_i64(w.gsize, w.gsize, nb + 1, w.gtotal, w.scan_ws, st);
    if (s != TB_OK) return s;
    pair_tasks_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(nb, w.gsize, w.key, w.fill, w.tasks);
    TB_CHECK_LAUNCH();
    return TB_OK;
  }

  static tb_status launch_pair(int64_t n, const int64_t *slice_ptr, const int32_t *col, const valT *val,
                               const valT *diag, real *P, real *Q, PairWs &w, int pair, real alpha, real shift,
                               int *flags, cudaStream_t st) {
    PairPlan plan = w.plan;
    double *bpart = w.bpart;
    void *args[] = {&n, &slice_ptr, &col, &val, &diag, &P, &Q, &plan, &pair, &bpart, &alpha, &shift, &flags};
    if (use_bulk()) {
      using GP = BulkGeom<real, valT, R, CPT, 1>;
      TB_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(cheb_pair_bulk_kernel<real, valT, R, CPT>),
                                          dim3(pair_grid()), dim3(kBlock), args, GP::kSmem, st));
    } else {
      TB_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(cheb_pair_kernel<real, valT, R, CPT>),
                                          dim3(pair_grid()), dim3(kBlock), args, 0, st));
    }
    note_launch();
    return TB_OK;
  }

  // The whole recursion: random phases, the Chebyshev steps, the reduction.
  template <bool SEG>
  static tb_status enqueue(int grid, int64_t n, const int64_t *slice_ptr, const int32_t *col, const valT *val,
                           const valT *diag, double a, double b, int M, uint64_t seed, int64_t r0, bool dbl,
                           double *mu_r, real *v0, real *A, real *B, double *partial, int *flags, const BatchTables &bt,
                           cudaStream_t st, cudaEvent_t ev_begin, cudaEvent_t ev_end, PairWs *pw = nullptr) {
    const int64_t units = SEG ? blocks(n) : grid;   // partials per moment slot
    const int64_t ps = units * R;
    TB_CUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
    random_phase_kernel<real, R, CPT, SEG><<<grid, kBlock, 0, st>>>(n, seed, r0, bt, v0, partial);
    TB_CHECK_LAUNCH();
    if (ev_begin) TB_CUDA(cudaEventRecord(ev_begin, st));
    // v1 = H~ v0 -> A.  Direct mode: the step making v_m adds the partials of
    // mu_m; doubling mode: the step reading v_k adds those of S_2k and S_2k+1.
    const real shift = static_cast<real>(b);
    const real inv_a = static_cast<real>(1.0 / a);
    tb_status s =
        dbl ? Kit::template step<true, true, SEG>(grid, n, slice_ptr, col, val, diag, v0, nullptr, v0, A, partial,
                                                  inv_a, shift, flags, ps, bt, st)
            : Kit::template step<true, false, SEG>(grid, n, slice_ptr, col, val, diag, v0, nullptr, v0, A,
                                                   partial + ps, inv_a, shift, flags, ps, bt, st);
    if (s != TB_OK) return s;
    const real two_over_a = static_cast<real>(2.0 / a);
    const int last = dbl ? (M - 1) / 2 + 1 : M - 1;   // index of the last vector computed
    auto single = [&](int m) {
      // v_m is written over v_{m-2}: m even -> B, m odd -> A; v_2 reads prev = v0
      real *out = (m & 1) ? A : B;
      const real *x = (m & 1) ? B : A;
      const real *prev = (m == 2) ? v0 : out;
      return dbl ? Kit::template step<false, true, SEG>(grid, n, slice_ptr, col, val, diag, x, prev, v0, out,
                                                        partial + (size_t)(2 * (m - 1)) * ps, two_over_a, shift,
                                                        flags, ps, bt, st)
                 : Kit::template step<false, false, SEG>(grid, n, slice_ptr, col, val, diag, x, prev, v0, out,
                                                         partial + (size_t)m * ps, two_over_a, shift, flags, ps,
                                                         bt, st);
    };
    int m = 2;
    if (!SEG && pw && last >= 4) {
      // v_2 alone (its v_{m-2} is v0), then v_m and v_{m+1} per launch
      s = single(2);
      if (s != TB_OK) return s;
      int pair = 0;
      for (m = 3; m + 1 <= last; m += 2, ++pair) {
        real *P = (m & 1) ? A : B;   // v_{m-2} -> v_m
        real *Q = (m & 1) ? B : A;   // v_{m-1} -> v_{m+1}
        s = launch_pair(n, slice_ptr, col, val, diag, P, Q, *pw, pair, two_over_a, shift, flags, st);
        if (s != TB_OK) return s;
        pair_reduce_kernel<<<(unsigned)((4 * units * R + 255) / 256), 256, 0, st>>>(
            pw->bpart, pw->plan.nb, R, (int)units, partial + (size_t)(2 * (m - 1)) * ps, ps);
        TB_CHECK_LAUNCH();
      }
    }
    for (; m <= last; ++m) {
      s = single(m);
      if (s != TB_OK) return s;
    }
    if (ev_end) TB_CUDA(cudaEventRecord(ev_end, st));
    if (SEG) {
      const int64_t total = (int64_t)bt.n_snap * M * R;
      batched_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(bt, M, R, RPB, units, partial,
                                                                             dbl ? 1 : 0, mu_r, flags);
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

  static tb_status run(int64_t n, const int64_t *slice_ptr, const int32_t *col, const valT *val, const valT *diag,
                       double a, double b, int M, uint64_t seed, int64_t r0, int mode, double *mu_r, void *ws,
                       size_t ws_bytes, cudaStream_t st, double *step_ms) {
    const bool dbl = mode == TB_KPM_DOUBLING;
    const int grid = grid_for(n, dbl);
    const int64_t np = padded_rows(n);
    Carver cv(ws, ws_bytes);
    real *v0 = cv.take<real>((size_t)np * R * 2);
    real *A = cv.take<real>((size_t)np * R * 2);
    real *B = cv.take<real>((size_t)np * R * 2);
    double *partial = cv.take<double>((size_t)(M + 1) * grid * R);
    int *flags = cv.take<int>(4);
    PairWs pw;
    carve_pair(cv, n, M, &pw);
    if (!cv.ok()) return fail(TB_ERR_WORKSPACE, "kpm_moments: workspace too small (%zu < %zu)", ws_bytes, cv.used);
    if (use_bulk() && ((reinterpret_cast<uintptr_t>(col) | reinterpret_cast<uintptr_t>(val)) & 15))
      return fail(TB_ERR_INVALID_ARG, "kpm_moments: col and val must be 16-byte aligned");
    prepare();
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (step_ms) {
      TB_CUDA(cudaEventCreate(&ev[0]));
      TB_CUDA(cudaEventCreate(&ev[1]));
    }
    const bool paired = use_pair(dbl);
    tb_status s = paired ? build_pair_plan(n, slice_ptr, col, pw, st) : TB_OK;
    if (s == TB_OK)
      s = enqueue<false>(grid, n, slice_ptr, col, val, diag, a, b, M, seed, r0, dbl, mu_r, v0, A, B, partial, flags,
                         BatchTables(), st, ev[0], ev[1], paired ? &pw : nullptr);
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

  // Batched: the caller's block-diagonal, already rescaled matrix of
  // n_pad rows (see kpm_moments_batched); the recursion is captured once as
  // a CUDA graph and launched on `st`.
  static tb_status run_batched(int64_t n_pad, const int64_t *slice_ptr, const int32_t *col, const valT *val,
                               const valT *diag, int M, uint64_t seed, int mode, const BatchTables &bt,
                               double *mu, void *ws, size_t ws_bytes, cudaStream_t st, double *graph_ms) {
    const bool dbl = mode == TB_KPM_DOUBLING;
    const int grid = grid_for(n_pad, dbl);
    Carver cv(ws, ws_bytes);
    real *v0 = cv.take<real>((size_t)n_pad * R * 2);
    real *A = cv.take<real>((size_t)n_pad * R * 2);
    real *B = cv.take<real>((size_t)n_pad * R * 2);
    double *partial = cv.take<double>((size_t)(M + 1) * blocks(n_pad) * R);
    int *flags = cv.take<int>(4);
    if (!cv.ok()) return fail(TB_ERR_WORKSPACE, "kpm_moments_batched: workspace too small");
    prepare();
    cudaStream_t cs = nullptr;
    TB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    tb_status s = TB_OK;
    if (e == cudaSuccess) {
      s = enqueue<true>(grid, n_pad, slice_ptr, col, val, diag, 1.0, 0.0, M, seed, 0, dbl, mu, v0, A, B, partial, flags,
                        bt, cs, nullptr, nullptr);
      e = cudaStreamEndCapture(cs, &graph);
    }
    if (e == cudaSuccess && s == TB_OK) e = cudaGraphInstantiate(&exec, graph, 0);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (e == cudaSuccess && s == TB_OK && graph_ms) {
      cudaEventCreate(&ev[0]);
      cudaEventCreate(&ev[1]);
      cudaEventRecord(ev[0], st);
    }
    if (e == cudaSuccess && s == TB_OK) e = cudaGraphLaunch(exec, st);
    if (ev[1]) cudaEventRecord(ev[1], st);
    if (e == cudaSuccess && s == TB_OK) s = check_flags(flags, st, "kpm_moments_batched");
    if (graph_ms && ev[1]) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[0], ev[1]);
      *graph_ms = ms;
    }
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(e, "kpm_moments_batched graph", __FILE__, __LINE__);
    return s;
  }
};

template <typename real, typename valT>
struct KpmDispatch {
  template <template <typename, typename, int> class Op, typename... Args>
  static bool call(int R, tb_status &st, Args... args) {
    switch (R) {
      case 1: st = Op<real, valT, 1>::apply(args...); return true;
      case 2: st = Op<real, valT, 2>::apply(args...); return true;
      case 4: st = Op<real, valT, 4>::apply(args...); return true;
      case 8: st = Op<real, valT, 8>::apply(args...); return true;
      case 16: st = Op<real, valT, 16>::apply(args...); return true;
      case 32: st = Op<real, valT, 32>::apply(args...); return true;
      default: return false;
    }
  }
};

// Copy snapshot s into the block-diagonal batch matrix with its rescaling
// folded in: val' = val / a_s, diag' = (diag - b_s) / a_s on the real rows
// (0 on padding rows); columns shifted by the snapshot's first row; padding
// slices get width 0.
template <typename valT>
__global__ void batch_fold_kernel(const int64_t *__restrict__ sp, const int32_t *__restrict__ col,
                                  const valT *__restrict__ val, const valT *__restrict__ diag, int64_t rows,
                                  int64_t n_slices, int64_t pad_slices, int64_t total, int64_t row0, int64_t e0,
                                  double inv_a, double shift, int64_t *__restrict__ dsp, int32_t *__restrict__ dcol,
                                  valT *__restrict__ dval, valT *__restrict__ ddiag) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t <= pad_slices) dsp[row0 / 32 + t] = e0 + (t <= n_slices ? sp[t] : total);
  if (t < total) {
    // rows >= `rows` of the last slice are phantom rows: value 0 whatever
    // the source holds there
    const int64_t last0 = n_slices > 0 ? sp[n_slices - 1] : 0;
    const bool phantom = t >= last0 && (n_slices - 1) * 32 + (t - last0) % 32 >= rows;
    dcol[e0 + t] = col[t] + static_cast<int32_t>(row0);
    dval[e0 + t] = phantom ? valT(0) : static_cast<valT>((double)val[t] * inv_a);
  }
  if (t < pad_slices * 32)
    ddiag[row0 + t] = t < rows ? static_cast<valT>(((diag ? (double)diag[t] : 0.0) - shift) * inv_a) : valT(0);
}

template <typename real, typename valT, int R>
struct BatchWsOp {
  static tb_status apply(int64_t n_pad, int M, size_t *out) {
    *out = KpmRunner<real, valT, R>::workspace(n_pad, M, true);
    return TB_OK;
  }
};

template <typename real, typename valT, int R>
struct BatchRunOp {
  static tb_status apply(int64_t n_pad, const int64_t *sp, const int32_t *col, const void *val, const void *diag,
                         int M, uint64_t seed, int mode, const BatchTables *bt, double *mu, void *ws, size_t wsb,
                         cudaStream_t st, double *ms) {
    return KpmRunner<real, valT, R>::run_batched(n_pad, sp, col, static_cast<const valT *>(val),
                                                 static_cast<const valT *>(diag), M, seed, mode, *bt, mu, ws, wsb, st,
                                                 ms);
  }
};

struct BatchLayout {
  int64_t n_pad = 0, elements = 0;
  std::vector<int64_t> row0, rows, e0, total, slices, pad_slices;
  std::vector<int32_t> tile_snap;
};

template <typename real, typename valT, int R>
struct WsOp {
  static tb_status apply(int64_t n, int M, size_t *out) {
    *out = KpmRunner<real, valT, R>::workspace(n, M, false);
    return TB_OK;
  }
};

template <typename real, typename valT, int R>
struct RunOp {
  static tb_status apply(int64_t n, const int64_t *sp, const int32_t *col, const void *val, const void *diag,
                         double a, double b, int M, uint64_t seed, int64_t r0, int mode, double *mu, void *ws,
                         size_t wsb, cudaStream_t st, double *step_ms) {
    return KpmRunner<real, valT, R>::run(n, sp, col, static_cast<const valT *>(val),
                                         static_cast<const valT *>(diag), a, b, M, seed, r0, mode, mu, ws, wsb, st,
                                         step_ms);
  }
};

}  // namespace
}  // namespace gputb

using namespace gputb;

extern "C" tb_status tb_kpm_set_variant(int32_t variant) {
  TB_REQUIRE(variant >= 0 && variant <= 3, "tb_kpm_set_variant: variant must be 0, 1, 2 or 3");
  g_kpm_variant = variant;
  return TB_OK;
}

extern "C" size_t kpm_moments_workspace_size(int64_t n, int32_t M, int32_t R, int32_t precision) {
  if (n <= 0 || M < 2) return 0;
  size_t out = 0;
  tb_status st = TB_OK;
  bool ok = precision == TB_F32 ? KpmDispatch<float, float>::call<WsOp>(R, st, n, (int)M, &out)
                                : KpmDispatch<double, double>::call<WsOp>(R, st, n, (int)M, &out);
  return ok ? out : 0;
}

extern "C" tb_status kpm_moments(int64_t n, const int64_t *slice_ptr, const int32_t *col, const void *val,
                                 const void *diag, int32_t precision, double a, double b, int32_t M, int32_t R,
                                 uint64_t seed, int64_t first_vector, int32_t mode, double *mu_r, void *workspace,
                                 size_t workspace_bytes, void *stream, double *step_ms) {
  TB_REQUIRE(first_vector >= 0 && first_vector <= (int64_t(1) << 31), "kpm_moments: first_vector out of range");
  TB_REQUIRE(mode == TB_KPM_DIRECT || mode == TB_KPM_DOUBLING, "kpm_moments: bad mode %d", mode);
  TB_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "kpm_moments: n=%lld out of range", (long long)n);
  TB_REQUIRE(M >= 2, "kpm_moments: M=%d must be >= 2", M);
  TB_REQUIRE(precision == TB_F32 || precision == TB_F64, "kpm_moments: bad precision %d", precision);
  TB_REQUIRE(a > 0.0 && std::isfinite(a) && std::isfinite(b), "kpm_moments: need finite a > 0, b");
  TB_REQUIRE(slice_ptr && mu_r && workspace, "kpm_moments: null pointer argument");
  TB_REQUIRE((reinterpret_cast<uintptr_t>(workspace) & 255) == 0, "kpm_moments: workspace must be 256-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tb_status status = TB_OK;
  bool ok = precision == TB_F32
                ? KpmDispatch<float, float>::call<RunOp>(R, status, n, slice_ptr, col, val, diag, a, b, (int)M,
                                                         seed, first_vector, (int)mode, mu_r, workspace,
                                                         workspace_bytes, st, step_ms)
                : KpmDispatch<double, double>::call<RunOp>(R, status, n, slice_ptr, col, val, diag, a, b, (int)M,
                                                           seed, first_vector, (int)mode, mu_r, workspace,
                                                           workspace_bytes, st, step_ms);
  if (!ok) return fail(TB_ERR_INVALID_ARG, "kpm_moments: unsupported R=%d for precision %d", R, precision);
  return status;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of kpm_moments.
//
// Some callers cannot allocate device memory at the point where they want
// the moments: code running inside a framework that owns the device memory
// pool and forbids outside allocations, real-time or latency-critical loops
// where cudaMalloc would synchronise the device, and plug-ins that only
// receive input and output buffers.  For them the scratch space (the three
// vector blocks, the per-CTA moment partials and the status flags) lives in
// one statically sized device array that the CUDA module carries; every GPU
// that loads this library holds it until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace gputb {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB limit
static __device__ __align__(256) unsigned char g_kpm_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
struct NoAllocSlot {
  std::once_flag once;
  void *ptr = nullptr;
  cudaError_t err = cudaSuccess;
};
NoAllocSlot g_noalloc_slots[kMaxDevices];

// Device address of the static scratch array on the current device.  In host
// code the array's name is only a host-side stand-in, so the address is
// looked up once per device with that device current.
tb_status noalloc_scratch(void **out) {
  int dev = 0;
  TB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(TB_ERR_INVALID_ARG, "kpm_moments_noalloc: device %d", dev);
  NoAllocSlot &slot = g_noalloc_slots[dev];
  std::call_once(slot.once, [&slot] {
    slot.err = cudaGetSymbolAddress(&slot.ptr, g_kpm_noalloc_scratch);
  });
  if (slot.err != cudaSuccess) return cuda_fail(slot.err, "cudaGetSymbolAddress", __FILE__, __LINE__);
  if (!slot.ptr) return fail(TB_ERR_CUDA, "kpm_moments_noalloc: null scratch address");
  *out = slot.ptr;
  return TB_OK;
}

}  // namespace
}  // namespace gputb

extern "C" tb_status kpm_moments_noalloc(int64_t n, const int64_t *slice_ptr, const int32_t *col, const void *val,
                                         const void *diag, int32_t precision, double a, double b, int32_t M,
                                         int32_t R, uint64_t seed, double *mu_r, void *stream) {
  TB_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "kpm_moments_noalloc: n=%lld out of range", (long long)n);
  TB_REQUIRE(M >= 2, "kpm_moments_noalloc: M=%d must be >= 2", M);
  TB_REQUIRE(precision == TB_F32 || precision == TB_F64, "kpm_moments_noalloc: bad precision %d", precision);
  TB_REQUIRE(a > 0.0 && std::isfinite(a) && std::isfinite(b), "kpm_moments_noalloc: need finite a > 0, b");
  TB_REQUIRE(slice_ptr && mu_r, "kpm_moments_noalloc: null pointer argument");
  const size_t need = kpm_moments_workspace_size(n, M, R, precision);
  if (need == 0) return fail(TB_ERR_INVALID_ARG, "kpm_moments_noalloc: unsupported R=%d", R);
  if (need > kNoAllocScratchBytes)
    return fail(TB_ERR_WORKSPACE,
                "kpm_moments_noalloc: this size needs %zu bytes of scratch but the built-in scratch holds %zu "
                "bytes (32 MiB); call kpm_moments with a caller workspace instead",
                need, kNoAllocScratchBytes);
  void *scratch = nullptr;
  tb_status status = noalloc_scratch(&scratch);
  if (status != TB_OK) return status;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the shared KPM runner clears the status flags it accumulates; every other
  // scratch word is written before it is read
  bool ok = precision == TB_F32
                ? KpmDispatch<float, float>::call<RunOp>(R, status, n, slice_ptr, col, val, diag, a, b, (int)M,
                                                         seed, (int64_t)0, (int)TB_KPM_DIRECT, mu_r, scratch,
                                                         kNoAllocScratchBytes, st, nullptr)
                : KpmDispatch<double, double>::call<RunOp>(R, status, n, slice_ptr, col, val, diag, a, b, (int)M,
                                                           seed, (int64_t)0, (int)TB_KPM_DIRECT, mu_r, scratch,
                                                           kNoAllocScratchBytes, st, nullptr);
  if (!ok) return fail(TB_ERR_INVALID_ARG, "kpm_moments_noalloc: unsupported R=%d", R);
  return status;
}

// ---------------------------------------------------------------------------
// Batched KPM over uneven snapshots (multi-frame averaging, Sec. 2.4).
// ---------------------------------------------------------------------------
namespace gputb {
namespace {

tb_status batch_layout(int n_snap, const int64_t *n_rows, const int64_t *const *slice_ptr, bool read_totals,
                       cudaStream_t st, BatchLayout *L) {
  L->row0.resize(n_snap);
  L->rows.resize(n_snap);
  L->e0.resize(n_snap);
  L->total.assign(n_snap, 0);
  L->slices.resize(n_snap);
  L->pad_slices.resize(n_snap);
  L->tile_snap.clear();
  int64_t row = 0, el = 0;
  for (int s = 0; s < n_snap; ++s) {
    TB_REQUIRE(n_rows[s] >= 1 && n_rows[s] < (int64_t(1) << 31), "kpm_moments_batched: snapshot %d size", s);
    const int64_t padded = (n_rows[s] + kBatchTile - 1) / kBatchTile * kBatchTile;
    L->row0[s] = row;
    L->rows[s] = n_rows[s];
    L->slices[s] = (n_rows[s] + 31) / 32;
    L->pad_slices[s] = padded / 32;
    if (read_totals) {
      TB_REQUIRE(slice_ptr && slice_ptr[s], "kpm_moments_batched: snapshot %d has no slice_ptr", s);
      TB_CUDA(cudaMemcpyAsync(&L->total[s], slice_ptr[s] + L->slices[s], sizeof(int64_t), cudaMemcpyDeviceToHost,
                              st));
    }
    for (int64_t q = 0; q < padded / kBatchTile; ++q) L->tile_snap.push_back(s);
    row += padded;
  }
  if (read_totals) TB_CUDA(cudaStreamSynchronize(st));
  for (int s = 0; s < n_snap; ++s) {
    L->e0[s] = el;
    el += L->total[s];
  }
  L->n_pad = row;
  L->elements = el;
  return TB_OK;
}

size_t batch_prefix_bytes(const BatchLayout &L, int n_snap, size_t val_size) {
  Carver cv(nullptr, 0);
  cv.take<int64_t>(L.n_pad / 32 + 1);
  cv.take<int32_t>(L.elements > 0 ? L.elements : 1);
  cv.take<char>((L.elements > 0 ? L.elements : 1) * val_size);
  cv.take<char>(L.n_pad * val_size);
  cv.take<int32_t>(L.tile_snap.size());
  cv.take<int64_t>(n_snap);
  cv.take<int64_t>(n_snap);
  return align_up(cv.used, 256);
}

}  // namespace
}  // namespace gputb

extern "C" size_t kpm_moments_batched_workspace_size(int32_t n_snap, const int64_t *const *slice_ptr,
                                                     const int64_t *n_rows, int32_t M, int32_t R,
                                                     int32_t precision, void *stream) {
  if (n_snap < 1 || !n_rows || !slice_ptr || M < 2) return 0;
  BatchLayout L;
  if (batch_layout(n_snap, n_rows, slice_ptr, true, static_cast<cudaStream_t>(stream), &L) != TB_OK) return 0;
  size_t run = 0;
  tb_status st = TB_OK;
  const bool ok = precision == TB_F32 ? KpmDispatch<float, float>::call<BatchWsOp>(R, st, L.n_pad, (int)M, &run)
                                      : KpmDispatch<double, double>::call<BatchWsOp>(R, st, L.n_pad, (int)M, &run);
  if (!ok) return 0;
  return batch_prefix_bytes(L, n_snap, precision == TB_F32 ? 4 : 8) + run + 256;
}

extern "C" tb_status kpm_moments_batched(int32_t n_snap, const int64_t *n_rows, const int64_t *const *slice_ptr,
                                         const int32_t *const *col, const void *const *val, const void *const *diag,
                                         int32_t precision, const double *a, const double *b, int32_t M, int32_t R,
                                         uint64_t seed, int32_t mode, double *mu, void *workspace,
                                         size_t workspace_bytes, void *stream, double *graph_ms) {
  TB_REQUIRE(n_snap >= 1 && n_rows && slice_ptr && col && val && a && b && mu && workspace,
             "kpm_moments_batched: bad argument");
  TB_REQUIRE(M >= 2, "kpm_moments_batched: M must be >= 2");
  TB_REQUIRE(precision == TB_F32 || precision == TB_F64, "kpm_moments_batched: bad precision");
  TB_REQUIRE(mode == TB_KPM_DIRECT || mode == TB_KPM_DOUBLING, "kpm_moments_batched: bad mode");
  TB_REQUIRE((reinterpret_cast<uintptr_t>(workspace) & 255) == 0, "kpm_moments_batched: workspace alignment");
  for (int s = 0; s < n_snap; ++s)
    TB_REQUIRE(a[s] > 0.0 && std::isfinite(a[s]) && std::isfinite(b[s]), "kpm_moments_batched: bad a/b of %d", s);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  BatchLayout L;
  tb_status status = batch_layout(n_snap, n_rows, slice_ptr, true, st, &L);
  if (status != TB_OK) return status;
  const size_t vs = precision == TB_F32 ? 4 : 8;
  Carver cv(workspace, workspace_bytes);
  int64_t *dsp = cv.take<int64_t>(L.n_pad / 32 + 1);
  int32_t *dcol = cv.take<int32_t>(L.elements > 0 ? L.elements : 1);
  char *dval = cv.take<char>((L.elements > 0 ? L.elements : 1) * vs);
  char *ddiag = cv.take<char>(L.n_pad * vs);
  int32_t *dtile = cv.take<int32_t>(L.tile_snap.size());
  int64_t *drow0 = cv.take<int64_t>(n_snap);
  int64_t *drows = cv.take<int64_t>(n_snap);
  cv.used = align_up(cv.used, 256);
  if (!cv.ok()) return fail(TB_ERR_WORKSPACE, "kpm_moments_batched: workspace too small");
  void *run_ws = static_cast<char *>(workspace) + cv.used;
  const size_t run_bytes = workspace_bytes - cv.used;
  TB_CUDA(cudaMemcpyAsync(dtile, L.tile_snap.data(), L.tile_snap.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                          st));
  TB_CUDA(cudaMemcpyAsync(drow0, L.row0.data(), n_snap * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  TB_CUDA(cudaMemcpyAsync(drows, L.rows.data(), n_snap * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  for (int s = 0; s < n_snap; ++s) {
    const int64_t work = std::max(L.total[s], L.pad_slices[s] * 32 + 1);
    const unsigned nb = (unsigned)((work + 255) / 256);
    if (precision == TB_F32)
      batch_fold_kernel<float><<<nb, 256, 0, st>>>(slice_ptr[s], col[s], static_cast<const float *>(val[s]),
                                                   diag ? static_cast<const float *>(diag[s]) : nullptr, L.rows[s],
                                                   L.slices[s], L.pad_slices[s], L.total[s], L.row0[s], L.e0[s],
                                                   1.0 / a[s], b[s], dsp, dcol, reinterpret_cast<float *>(dval),
                                                   reinterpret_cast<float *>(ddiag));
    else
      batch_fold_kernel<double><<<nb, 256, 0, st>>>(slice_ptr[s], col[s], static_cast<const double *>(val[s]),
                                                    diag ? static_cast<const double *>(diag[s]) : nullptr,
                                                    L.rows[s], L.slices[s], L.pad_slices[s], L.total[s], L.row0[s],
                                                    L.e0[s], 1.0 / a[s], b[s], dsp, dcol,
                                                    reinterpret_cast<double *>(dval),
                                                    reinterpret_cast<double *>(ddiag));
    TB_CHECK_LAUNCH();
  }
  TB_CUDA(cudaStreamSynchronize(st));  // the host tables above may go out of scope
  BatchTables bt;
  bt.tile_snap = dtile;
  bt.row0 = drow0;
  bt.rows = drows;
  bt.n_snap = n_snap;
  const bool ok = precision == TB_F32
                      ? KpmDispatch<float, float>::call<BatchRunOp>(R, status, L.n_pad, (const int64_t *)dsp,
                                                                    (const int32_t *)dcol, (const void *)dval,
                                                                    (const void *)ddiag, (int)M, seed, (int)mode, &bt,
                                                                    mu, run_ws, run_bytes, st, graph_ms)
                      : KpmDispatch<double, double>::call<BatchRunOp>(R, status, L.n_pad, (const int64_t *)dsp,
                                                                      (const int32_t *)dcol, (const void *)dval,
                                                                      (const void *)ddiag, (int)M, seed, (int)mode,
                                                                      &bt, mu, run_ws, run_bytes, st, graph_ms);
  if (!ok) return fail(TB_ERR_INVALID_ARG, "kpm_moments_batched: unsupported R=%d", R);
  return status;
}

// ---------------------------------------------------------------------------
// Test hook for failure handling: the same bounded waits that the pipelined
// step (mbarrier phase) and the two-step kernel (stage-1 flags) use, run on
// a barrier phase or flags that nothing completes, must give up after
// `polls` polls and report, leaving the context usable.
// ---------------------------------------------------------------------------
namespace gputb {
namespace {

__global__ void wait_probe_kernel(int which, long long polls, PairPlan plan, int *__restrict__ status) {
  __shared__ unsigned long long s_tot;
  __shared__ __align__(8) uint64_t bar;
  bool ok;
  if (which == 0) {
    ok = pair_wait(plan, make_int2(0, 63), 1, 0, polls, &s_tot);   // flags stay 0, epoch 1
  } else {
    if (threadIdx.x == 0) mbar_init(&bar, 1);                       // one arrival expected, none made
    __syncthreads();
    ok = __syncthreads_and(mbar_wait_bounded(&bar, 0, polls)) != 0;
  }
  if (threadIdx.x == 0) *status = ok ? 1 : 0;
}

}  // namespace
}  // namespace gputb

extern "C" tb_status tb_debug_wait_timeout(int32_t which, int64_t polls, void *workspace, size_t workspace_bytes,
                                           void *stream) {
  TB_REQUIRE(which == 0 || which == 1, "tb_debug_wait_timeout: which must be 0 (flags) or 1 (mbarrier)");
  TB_REQUIRE(polls >= 1 && polls <= (int64_t(1) << 24), "tb_debug_wait_timeout: polls out of range");
  TB_REQUIRE(workspace && workspace_bytes >= 512, "tb_debug_wait_timeout: need 512 bytes of workspace");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int *done = static_cast<int *>(workspace);   // 64 flags, then the status word
  TB_CUDA(cudaMemsetAsync(done, 0, 512, st));
  PairPlan plan;
  plan.done = done;
  plan.cta_s1 = done;
  plan.nb = 64;
  wait_probe_kernel<<<1, kBlock, 0, st>>>(which, (long long)polls, plan, done + 64);
  TB_CHECK_LAUNCH();
  int h = -1;
  TB_CUDA(cudaMemcpyAsync(&h, done + 64, sizeof(int), cudaMemcpyDeviceToHost, st));
  TB_CUDA(cudaStreamSynchronize(st));
  if (h == 0) return fail(TB_ERR_TIMEOUT, "tb_debug_wait_timeout: the %s wait gave up after %lld polls",
                          which == 0 ? "flag" : "mbarrier", (long long)polls);
  return TB_OK;
}
