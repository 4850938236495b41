// Precision-specific KPM runners behind the C ABI of kpm.cu.  Each is
// defined twice, for complex FP32 vectors with FP32 matrix values
// (kpm_f32.cu) and for complex FP64 vectors with FP64 values (kpm_f64.cu), so
// that the two sets of step-kernel instantiations compile in parallel.  Every
// function returns false when R is not one of 1, 2, 4, 8, 16, 32 (and then
// leaves its outputs untouched).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "gputb.h"

namespace gputb {
namespace kpmdev {

// Device tables of a block-diagonal batch (kpm_moments_batched).
struct BatchDesc {
  const int32_t *tile_snap;   // snapshot of each 256-row tile
  const int64_t *row0;        // first row of each snapshot
  const int64_t *rows;        // real rows of each snapshot
  int n_snap;
};

template <typename real>
struct KpmEntry {
  // candidate step shapes for R (see Shapes in kpm_step.cuh)
  static bool shape_count(int R, int *count);
  static bool shape_info(int R, int shape, tb_step_shape *out);
  // CTAs of one step launch of `shape` over n rows (occupancy query)
  static bool shape_grid(int R, int shape, int64_t n, bool doubling, int *out);
  // workspace of kpm_moments (segmented = the batched layout of n rows)
  static bool workspace(int R, int64_t n, int M, bool segmented, size_t *out);
  static bool run(int R, tb_status *status, int shape, int64_t n, const int64_t *slice_ptr, const int32_t *col,
                  const void *val, const void *diag, double a, double b, int M, uint64_t seed, int64_t r0,
                  int mode, double *mu_r, void *ws, size_t ws_bytes, cudaStream_t st, double *step_ms);
  // opt the shape's kernels into their shared memory (before any capture)
  static bool prepare(int R, int shape);
  // enqueue the batched recursion on `st` (capturable); *flags receives the
  // device status flags to check after it ran
  static bool enqueue_batched(int R, tb_status *status, int shape, int64_t n_pad, const int64_t *slice_ptr,
                              const int32_t *col, const void *val, const void *diag, int M, uint64_t seed, int mode,
                              const BatchDesc &bt, double *mu, void *ws, size_t ws_bytes, cudaStream_t st,
                              int **flags);
  // time `reps` Chebyshev steps of every candidate shape on this matrix;
  // ms[shape] receives the mean time per step, *best the fastest shape.
  // bt != nullptr: the segmented step of that block-diagonal batch
  static bool autotune(int R, tb_status *status, int64_t n, const int64_t *slice_ptr, const int32_t *col,
                       const void *val, const void *diag, double a, double b, int mode, int reps, void *ws,
                       size_t ws_bytes, cudaStream_t st, int *best, float *ms, int ms_capacity,
                       const BatchDesc *bt = nullptr);
};

}  // namespace kpmdev
}  // namespace gputb
