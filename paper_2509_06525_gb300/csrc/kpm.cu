// C ABI of the KPM moments: kpm_moments (single matrix), kpm_moments_noalloc
// (static scratch), kpm_moments_batched (many uneven snapshots in one CUDA
// graph), the table of step shapes and its autotuner.  The kernels and the
// recursion live in kpm_runner.cuh / kpm_step.cuh and are instantiated per
// precision in kpm_f32.cu and kpm_f64.cu.
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "kpm_entry.h"
#include "kpm_step.cuh"

// ---------------------------------------------------------------------------
// The shape table.  Entries are keyed by (precision, R, mode, size class)
// with size class floor(log2 n); class -1 forces a shape for every size.
// ---------------------------------------------------------------------------
namespace gputb {
namespace kpmdev {
namespace {
std::mutex g_shape_mu;
std::map<std::array<int, 4>, int> g_shape_table;

int size_class(int64_t n) {
  int c = 0;
  while (c < 62 && (int64_t(2) << c) <= n) ++c;
  return c;
}

bool shape_count(int precision, int R, int *count) {
  return precision == TB_F32 ? KpmEntry<float>::shape_count(R, count)
                             : KpmEntry<double>::shape_count(R, count);
}
}  // namespace

int chosen_shape(int precision, int R, int mode, int64_t n) {
  std::lock_guard<std::mutex> lock(g_shape_mu);
  auto it = g_shape_table.find({precision, R, mode, -1});
  if (it != g_shape_table.end()) return it->second;
  it = g_shape_table.find({precision, R, mode, size_class(n)});
  return it != g_shape_table.end() ? it->second : 0;
}
}  // namespace kpmdev
}  // namespace gputb

using namespace gputb;
using namespace gputb::kpmdev;

extern "C" int32_t tb_kpm_shape_count(int32_t R, int32_t precision) {
  if (precision != TB_F32 && precision != TB_F64) return 0;
  int c = 0;
  return shape_count(precision, R, &c) ? c : 0;
}

extern "C" tb_status tb_kpm_shape_info(int32_t R, int32_t precision, int32_t shape, tb_step_shape *out) {
  TB_REQUIRE(out, "tb_kpm_shape_info: null output");
  TB_REQUIRE(precision == TB_F32 || precision == TB_F64, "tb_kpm_shape_info: bad precision %d", precision);
  const bool ok = precision == TB_F32 ? KpmEntry<float>::shape_info(R, shape, out)
                                      : KpmEntry<double>::shape_info(R, shape, out);
  TB_REQUIRE(ok, "tb_kpm_shape_info: no shape %d for R=%d", shape, R);
  return TB_OK;
}

extern "C" tb_status tb_kpm_set_shape(int64_t n, int32_t R, int32_t precision, int32_t mode, int32_t shape) {
  TB_REQUIRE(precision == TB_F32 || precision == TB_F64, "tb_kpm_set_shape: bad precision %d", precision);
  TB_REQUIRE(mode == -1 || mode == TB_KPM_DIRECT || mode == TB_KPM_DOUBLING, "tb_kpm_set_shape: bad mode %d", mode);
  TB_REQUIRE(n >= 0, "tb_kpm_set_shape: n must be >= 0");
  const int count = tb_kpm_shape_count(R, precision);
  TB_REQUIRE(count > 0, "tb_kpm_set_shape: unsupported R=%d", R);
  TB_REQUIRE(shape >= -1 && shape < count, "tb_kpm_set_shape: shape %d out of range [-1, %d)", shape, count);
  std::lock_guard<std::mutex> lock(g_shape_mu);
  const int cls = n == 0 ? -1 : size_class(n);
  for (int m = 0; m < 2; ++m) {
    if (mode != -1 && mode != m) continue;
    const std::array<int, 4> key{precision, R, m, cls};
    if (shape < 0) g_shape_table.erase(key);
    else g_shape_table[key] = shape;
  }
  return TB_OK;
}

extern "C" tb_status tb_kpm_clear_shapes(void) {
  std::lock_guard<std::mutex> lock(g_shape_mu);
  g_shape_table.clear();
  return TB_OK;
}

extern "C" int32_t tb_kpm_get_shape(int64_t n, int32_t R, int32_t precision, int32_t mode) {
  if (tb_kpm_shape_count(R, precision) == 0 || n < 1) return -1;
  if (mode != TB_KPM_DIRECT && mode != TB_KPM_DOUBLING) return -1;
  return chosen_shape(precision, R, mode, n);
}

extern "C" int32_t tb_kpm_shape_grid(int64_t n, int32_t R, int32_t precision, int32_t mode, int32_t shape) {
  if (n < 1 || (precision != TB_F32 && precision != TB_F64)) return -1;
  if (mode != TB_KPM_DIRECT && mode != TB_KPM_DOUBLING) return -1;
  int g = -1;
  const bool dbl = mode == TB_KPM_DOUBLING;
  const bool ok = precision == TB_F32 ? KpmEntry<float>::shape_grid(R, shape, n, dbl, &g)
                                      : KpmEntry<double>::shape_grid(R, shape, n, dbl, &g);
  return ok ? g : -1;
}

extern "C" size_t kpm_moments_workspace_size(int64_t n, int32_t M, int32_t R, int32_t precision) {
  if (n <= 0 || M < 2) return 0;
  size_t out = 0;
  bool ok = false;
  if (precision == TB_F32) ok = KpmEntry<float>::workspace(R, n, M, false, &out);
  else if (precision == TB_F64) ok = KpmEntry<double>::workspace(R, n, M, false, &out);
  return ok ? out : 0;
}

namespace {
tb_status check_kpm_args(const char *who, int64_t n, const int64_t *slice_ptr, int32_t precision, double a,
                         double b, int32_t M) {
  TB_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "%s: n=%lld out of range", who, (long long)n);
  TB_REQUIRE(M >= 2, "%s: M=%d must be >= 2", who, M);
  TB_REQUIRE(precision == TB_F32 || precision == TB_F64, "%s: bad precision %d", who, precision);
  TB_REQUIRE(a > 0.0 && std::isfinite(a) && std::isfinite(b), "%s: need finite a > 0, b", who);
  TB_REQUIRE(slice_ptr, "%s: null slice_ptr", who);
  return TB_OK;
}

tb_status run_single(int64_t n, const int64_t *slice_ptr, const int32_t *col, const void *val, const void *diag,
                     int32_t precision, double a, double b, int32_t M, int32_t R, uint64_t seed,
                     int64_t first_vector, int32_t mode, double *mu_r, void *workspace, size_t workspace_bytes,
                     cudaStream_t st, double *step_ms, const char *who) {
  const int shape = chosen_shape(precision, R, mode, n);
  tb_status status = TB_OK;
  const bool ok = precision == TB_F32
                      ? KpmEntry<float>::run(R, &status, shape, n, slice_ptr, col, val, diag, a, b, (int)M, seed,
                                             first_vector, (int)mode, mu_r, workspace, workspace_bytes, st, step_ms)
                      : KpmEntry<double>::run(R, &status, shape, n, slice_ptr, col, val, diag, a, b, (int)M, seed,
                                              first_vector, (int)mode, mu_r, workspace, workspace_bytes, st,
                                              step_ms);
  if (!ok) return fail(TB_ERR_INVALID_ARG, "%s: unsupported R=%d for precision %d", who, R, precision);
  return status;
}
}  // namespace

extern "C" tb_status kpm_moments(int64_t n, const int64_t *slice_ptr, const int32_t *col, const void *val,
                                 const void *diag, int32_t precision, double a, double b, int32_t M, int32_t R,
                                 uint64_t seed, int64_t first_vector, int32_t mode, double *mu_r, void *workspace,
                                 size_t workspace_bytes, void *stream, double *step_ms) {
  tb_status s = check_kpm_args("kpm_moments", n, slice_ptr, precision, a, b, M);
  if (s != TB_OK) return s;
  TB_REQUIRE(first_vector >= 0 && first_vector <= (int64_t(1) << 31), "kpm_moments: first_vector out of range");
  TB_REQUIRE(mode == TB_KPM_DIRECT || mode == TB_KPM_DOUBLING, "kpm_moments: bad mode %d", mode);
  TB_REQUIRE(mu_r && workspace, "kpm_moments: null pointer argument");
  TB_REQUIRE((reinterpret_cast<uintptr_t>(workspace) & 255) == 0, "kpm_moments: workspace must be 256-byte aligned");
  return run_single(n, slice_ptr, col, val, diag, precision, a, b, M, R, seed, first_vector, mode, mu_r, workspace,
                    workspace_bytes, static_cast<cudaStream_t>(stream), step_ms, "kpm_moments");
}

extern "C" tb_status tb_kpm_autotune(int64_t n, const int64_t *slice_ptr, const int32_t *col, const void *val,
                                     const void *diag, int32_t precision, double a, double b, int32_t R,
                                     int32_t mode, int32_t reps, void *workspace, size_t workspace_bytes,
                                     void *stream, int32_t *best_shape, float *ms_per_step,
                                     int32_t ms_capacity) {
  tb_status s = check_kpm_args("tb_kpm_autotune", n, slice_ptr, precision, a, b, 2);
  if (s != TB_OK) return s;
  TB_REQUIRE(mode == TB_KPM_DIRECT || mode == TB_KPM_DOUBLING, "tb_kpm_autotune: bad mode %d", mode);
  TB_REQUIRE(reps >= 1 && reps <= 10000, "tb_kpm_autotune: reps=%d out of range [1, 10000]", reps);
  TB_REQUIRE(workspace && best_shape, "tb_kpm_autotune: null pointer argument");
  TB_REQUIRE(ms_capacity >= 0 && (ms_capacity == 0 || ms_per_step), "tb_kpm_autotune: bad ms_per_step buffer");
  TB_REQUIRE((reinterpret_cast<uintptr_t>(workspace) & 255) == 0, "tb_kpm_autotune: workspace alignment");
  int best = 0;
  tb_status status = TB_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool ok = precision == TB_F32
                      ? KpmEntry<float>::autotune(R, &status, n, slice_ptr, col, val, diag, a, b, (int)mode, (int)reps,
                                                  workspace, workspace_bytes, st, &best, ms_per_step, ms_capacity)
                      : KpmEntry<double>::autotune(R, &status, n, slice_ptr, col, val, diag, a, b, (int)mode,
                                                   (int)reps, workspace, workspace_bytes, st, &best, ms_per_step,
                                                   ms_capacity);
  if (!ok) return fail(TB_ERR_INVALID_ARG, "tb_kpm_autotune: unsupported R=%d", R);
  if (status != TB_OK) return status;
  *best_shape = best;
  return tb_kpm_set_shape(n, R, precision, mode, best);
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
  tb_status s = check_kpm_args("kpm_moments_noalloc", n, slice_ptr, precision, a, b, M);
  if (s != TB_OK) return s;
  TB_REQUIRE(mu_r, "kpm_moments_noalloc: null pointer argument");
  const size_t need = kpm_moments_workspace_size(n, M, R, precision);
  if (need == 0) return fail(TB_ERR_INVALID_ARG, "kpm_moments_noalloc: unsupported R=%d", R);
  if (need > kNoAllocScratchBytes)
    return fail(TB_ERR_WORKSPACE,
                "kpm_moments_noalloc: this size needs %zu bytes of scratch but the built-in scratch holds %zu "
                "bytes (32 MiB); call kpm_moments with a caller workspace instead",
                need, kNoAllocScratchBytes);
  void *scratch = nullptr;
  s = noalloc_scratch(&scratch);
  if (s != TB_OK) return s;
  // the shared KPM runner clears the status flags it accumulates; every other
  // scratch word is written before it is read
  return run_single(n, slice_ptr, col, val, diag, precision, a, b, M, R, seed, 0, TB_KPM_DIRECT, mu_r, scratch,
                    kNoAllocScratchBytes, static_cast<cudaStream_t>(stream), nullptr, "kpm_moments_noalloc");
}

// ---------------------------------------------------------------------------
// Batched KPM over uneven snapshots (multi-frame averaging, Sec. 2.4).
// ---------------------------------------------------------------------------
namespace gputb {
namespace {

constexpr int kBatchTileRows = 256;   // snapshots padded to whole 256-row tiles

struct BatchLayout {
  int64_t n_pad = 0, elements = 0;
  std::vector<int64_t> row0, rows, e0, total, slices, pad_slices;
  std::vector<int32_t> tile_snap;
};

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
    const int64_t padded = (n_rows[s] + kBatchTileRows - 1) / kBatchTileRows * kBatchTileRows;
    L->row0[s] = row;
    L->rows[s] = n_rows[s];
    L->slices[s] = (n_rows[s] + 31) / 32;
    L->pad_slices[s] = padded / 32;
    if (read_totals) {
      TB_REQUIRE(slice_ptr && slice_ptr[s], "kpm_moments_batched: snapshot %d has no slice_ptr", s);
      TB_CUDA(cudaMemcpyAsync(&L->total[s], slice_ptr[s] + L->slices[s], sizeof(int64_t), cudaMemcpyDeviceToHost,
                              st));
    }
    for (int64_t q = 0; q < padded / kBatchTileRows; ++q) L->tile_snap.push_back(s);
    row += padded;
  }
  TB_REQUIRE(row < (int64_t(1) << 31), "kpm_moments_batched: %lld padded rows in all (must be < 2^31)",
             (long long)row);
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

}  // namespace
}  // namespace gputb

extern "C" size_t kpm_moments_batched_workspace_size(int32_t n_snap, const int64_t *const *slice_ptr,
                                                     const int64_t *n_rows, int32_t M, int32_t R,
                                                     int32_t precision, void *stream) {
  if (n_snap < 1 || !n_rows || !slice_ptr || M < 2) return 0;
  if (precision != TB_F32 && precision != TB_F64) return 0;
  BatchLayout L;
  if (batch_layout(n_snap, n_rows, slice_ptr, true, static_cast<cudaStream_t>(stream), &L) != TB_OK) return 0;
  size_t run = 0;
  const bool ok = precision == TB_F32 ? KpmEntry<float>::workspace(R, L.n_pad, (int)M, true, &run)
                                      : KpmEntry<double>::workspace(R, L.n_pad, (int)M, true, &run);
  if (!ok) return 0;
  return batch_prefix_bytes(L, n_snap, precision == TB_F32 ? 4 : 8) + run + 256;
}

namespace gputb {
namespace {

// Checks shared by the batched entry points.
tb_status check_batch_args(const char *who, int32_t n_snap, const int64_t *n_rows, const int64_t *const *slice_ptr,
                           const int32_t *const *col, const void *const *val, int32_t precision, const double *a,
                           const double *b, int32_t R, int32_t mode, void *workspace) {
  TB_REQUIRE(n_snap >= 1 && n_rows && slice_ptr && col && val && a && b && workspace, "%s: bad argument", who);
  TB_REQUIRE(precision == TB_F32 || precision == TB_F64, "%s: bad precision", who);
  TB_REQUIRE(mode == TB_KPM_DIRECT || mode == TB_KPM_DOUBLING, "%s: bad mode", who);
  TB_REQUIRE((reinterpret_cast<uintptr_t>(workspace) & 255) == 0, "%s: workspace alignment", who);
  TB_REQUIRE(tb_kpm_shape_count(R, precision) > 0, "%s: unsupported R=%d", who, R);
  for (int s = 0; s < n_snap; ++s)
    TB_REQUIRE(a[s] > 0.0 && std::isfinite(a[s]) && std::isfinite(b[s]), "%s: bad a/b of snapshot %d", who, s);
  return TB_OK;
}

// The batch matrix in the workspace: pointers carved in a fixed order.
struct FoldedBatch {
  int64_t *sp = nullptr;
  int32_t *col = nullptr;
  char *val = nullptr;
  char *diag = nullptr;
  int32_t *tile = nullptr;
  int64_t *row0 = nullptr;
  int64_t *rows = nullptr;
  void *run_ws = nullptr;
  size_t run_bytes = 0;
};

tb_status carve_folded(const BatchLayout &L, int n_snap, size_t vs, void *workspace, size_t workspace_bytes,
                       FoldedBatch *F) {
  Carver cv(workspace, workspace_bytes);
  F->sp = cv.take<int64_t>(L.n_pad / 32 + 1);
  F->col = cv.take<int32_t>(L.elements > 0 ? L.elements : 1);
  F->val = cv.take<char>((L.elements > 0 ? L.elements : 1) * vs);
  F->diag = cv.take<char>(L.n_pad * vs);
  F->tile = cv.take<int32_t>(L.tile_snap.size());
  F->row0 = cv.take<int64_t>(n_snap);
  F->rows = cv.take<int64_t>(n_snap);
  cv.used = align_up(cv.used, 256);
  if (!cv.ok()) return fail(TB_ERR_WORKSPACE, "kpm_moments_batched: workspace too small");
  F->run_ws = static_cast<char *>(workspace) + cv.used;
  F->run_bytes = workspace_bytes - cv.used;
  return TB_OK;
}

// the layout tables to the device (on `st`)
tb_status upload_tables(const BatchLayout &L, int n_snap, const FoldedBatch &F, cudaStream_t st) {
  TB_CUDA(cudaMemcpyAsync(F.tile, L.tile_snap.data(), L.tile_snap.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                          st));
  TB_CUDA(cudaMemcpyAsync(F.row0, L.row0.data(), n_snap * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  TB_CUDA(cudaMemcpyAsync(F.rows, L.rows.data(), n_snap * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  return TB_OK;
}

// every snapshot into the block-diagonal matrix with its rescaling folded in
tb_status enqueue_fold(const BatchLayout &L, int n_snap, const int64_t *const *slice_ptr, const int32_t *const *col,
                       const void *const *val, const void *const *diag, int32_t precision, const double *a,
                       const double *b, const FoldedBatch &F, cudaStream_t st) {
  for (int s = 0; s < n_snap; ++s) {
    const int64_t work = std::max(L.total[s], L.pad_slices[s] * 32 + 1);
    const unsigned nb = (unsigned)((work + 255) / 256);
    if (precision == TB_F32)
      batch_fold_kernel<float><<<nb, 256, 0, st>>>(slice_ptr[s], col[s], static_cast<const float *>(val[s]),
                                                   diag ? static_cast<const float *>(diag[s]) : nullptr, L.rows[s],
                                                   L.slices[s], L.pad_slices[s], L.total[s], L.row0[s], L.e0[s],
                                                   1.0 / a[s], b[s], F.sp, F.col, reinterpret_cast<float *>(F.val),
                                                   reinterpret_cast<float *>(F.diag));
    else
      batch_fold_kernel<double><<<nb, 256, 0, st>>>(slice_ptr[s], col[s], static_cast<const double *>(val[s]),
                                                    diag ? static_cast<const double *>(diag[s]) : nullptr,
                                                    L.rows[s], L.slices[s], L.pad_slices[s], L.total[s], L.row0[s],
                                                    L.e0[s], 1.0 / a[s], b[s], F.sp, F.col,
                                                    reinterpret_cast<double *>(F.val),
                                                    reinterpret_cast<double *>(F.diag));
    TB_CHECK_LAUNCH();
  }
  return TB_OK;
}

// One instantiated graph (fold + recursion + reduction) of the last batched
// call, reused while every argument that its kernels see is the same.
struct BatchGraph {
  std::vector<uint64_t> key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int *flags = nullptr;
  int launches = 0;
};
std::mutex g_batch_mu;
BatchGraph g_batch_graph;

void batch_key(std::vector<uint64_t> &k, int device, int32_t n_snap, const BatchLayout &L,
               const int64_t *const *slice_ptr, const int32_t *const *col, const void *const *val,
               const void *const *diag, int32_t precision, const double *a, const double *b, int32_t M, int32_t R,
               uint64_t seed, int32_t mode, int shape, const double *mu, const void *ws, size_t wsb) {
  auto put = [&](uint64_t v) { k.push_back(v); };
  auto ptr = [&](const void *p) { put(reinterpret_cast<uintptr_t>(p)); };
  auto dbl = [&](double d) {
    uint64_t u;
    std::memcpy(&u, &d, 8);
    put(u);
  };
  put(device), put(n_snap), put(precision), put(M), put(R), put(seed), put(mode), put(shape);
  ptr(mu), ptr(ws), put(wsb);
  for (int s = 0; s < n_snap; ++s) {
    ptr(slice_ptr[s]), ptr(col[s]), ptr(val[s]), ptr(diag ? diag[s] : nullptr);
    put(L.rows[s]), put(L.total[s]);
    dbl(a[s]), dbl(b[s]);
  }
}

tb_status batch_flags_check(const int *flags, cudaStream_t st) {
  int h[4] = {0, 0, 0, 0};
  TB_CUDA(cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, st));
  TB_CUDA(cudaStreamSynchronize(st));
  if (h[0] & 4) return fail(TB_ERR_TIMEOUT, "kpm_moments_batched: a pipeline wait timed out");
  if (h[0] & 2) return fail(TB_ERR_NOT_FINITE, "kpm_moments_batched: non-finite moment");
  if (h[0] & 1)
    return fail(TB_ERR_BOUNDS, "kpm_moments_batched: |mu_n| > 1 + 1e-6; a spectrum is not inside [b - a, b + a]");
  return TB_OK;
}

}  // namespace
}  // namespace gputb

extern "C" tb_status kpm_moments_batched(int32_t n_snap, const int64_t *n_rows, const int64_t *const *slice_ptr,
                                         const int32_t *const *col, const void *const *val, const void *const *diag,
                                         int32_t precision, const double *a, const double *b, int32_t M, int32_t R,
                                         uint64_t seed, int32_t mode, double *mu, void *workspace,
                                         size_t workspace_bytes, void *stream, double *graph_ms) {
  tb_status status =
      check_batch_args("kpm_moments_batched", n_snap, n_rows, slice_ptr, col, val, precision, a, b, R, mode, workspace);
  if (status != TB_OK) return status;
  TB_REQUIRE(mu && M >= 2, "kpm_moments_batched: need mu and M >= 2");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  BatchLayout L;
  status = batch_layout(n_snap, n_rows, slice_ptr, true, st, &L);
  if (status != TB_OK) return status;
  const size_t vs = precision == TB_F32 ? 4 : 8;
  FoldedBatch F;
  status = carve_folded(L, n_snap, vs, workspace, workspace_bytes, &F);
  if (status != TB_OK) return status;
  const int shape = chosen_shape(precision, R, mode, L.n_pad);
  const bool prep = precision == TB_F32 ? KpmEntry<float>::prepare(R, shape) : KpmEntry<double>::prepare(R, shape);
  if (!prep) return fail(TB_ERR_INVALID_ARG, "kpm_moments_batched: bad shape %d for R=%d", shape, R);
  int device = 0;
  TB_CUDA(cudaGetDevice(&device));
  std::vector<uint64_t> key;
  batch_key(key, device, n_snap, L, slice_ptr, col, val, diag, precision, a, b, M, R, seed, mode, shape, mu,
            workspace, workspace_bytes);

  std::lock_guard<std::mutex> lock(g_batch_mu);
  BatchGraph &G = g_batch_graph;
  if (G.exec == nullptr || G.key != key) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    G = BatchGraph();
    // capture on a private stream: the fold of every snapshot, the band plan
    // (banded shapes), the random phases, the recursion and the reduction
    cudaStream_t cs = nullptr;
    TB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const int64_t l0 = tb_launch_count();
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int *flags = nullptr;
    if (e == cudaSuccess) {
      status = enqueue_fold(L, n_snap, slice_ptr, col, val, diag, precision, a, b, F, cs);
      BatchDesc bd{F.tile, F.row0, F.rows, n_snap};
      bool ok = true;
      if (status == TB_OK)
        ok = precision == TB_F32
                 ? KpmEntry<float>::enqueue_batched(R, &status, shape, L.n_pad, F.sp, F.col, F.val, F.diag, (int)M,
                                                    seed, (int)mode, bd, mu, F.run_ws, F.run_bytes, cs, &flags)
                 : KpmEntry<double>::enqueue_batched(R, &status, shape, L.n_pad, F.sp, F.col, F.val, F.diag,
                                                     (int)M, seed, (int)mode, bd, mu, F.run_ws, F.run_bytes, cs,
                                                     &flags);
      if (!ok && status == TB_OK) status = fail(TB_ERR_INVALID_ARG, "kpm_moments_batched: unsupported R=%d", R);
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(cs, &graph);
      G.graph = graph;
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(e, "kpm_moments_batched capture", __FILE__, __LINE__);
    if (status != TB_OK) return status;
    e = cudaGraphInstantiate(&G.exec, G.graph, 0);
    if (e != cudaSuccess) {
      G.exec = nullptr;
      return cuda_fail(e, "kpm_moments_batched graph", __FILE__, __LINE__);
    }
    G.key = key;
    G.flags = flags;
    G.launches = static_cast<int>(tb_launch_count() - l0);
    note_launches(-G.launches);   // captured, not yet run: counted at each graph launch below
  }
  // the tables the graph's kernels read, then the graph itself
  status = upload_tables(L, n_snap, F, st);
  if (status != TB_OK) return status;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (graph_ms) {
    TB_CUDA(cudaEventCreate(&ev[0]));
    TB_CUDA(cudaEventCreate(&ev[1]));
    TB_CUDA(cudaEventRecord(ev[0], st));
  }
  cudaError_t e = cudaGraphLaunch(G.exec, st);
  if (e == cudaSuccess) note_launches(G.launches);
  if (e == cudaSuccess && graph_ms) e = cudaEventRecord(ev[1], st);
  if (e == cudaSuccess) status = batch_flags_check(G.flags, st);
  if (graph_ms) {
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, ev[0], ev[1]);
    *graph_ms = ms;
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
  }
  if (e != cudaSuccess) return cuda_fail(e, "kpm_moments_batched launch", __FILE__, __LINE__);
  return status;
}

extern "C" tb_status kpm_moments_batched_autotune(int32_t n_snap, const int64_t *n_rows,
                                                  const int64_t *const *slice_ptr, const int32_t *const *col,
                                                  const void *const *val, const void *const *diag,
                                                  int32_t precision, const double *a, const double *b, int32_t R,
                                                  int32_t mode, int32_t reps, void *workspace,
                                                  size_t workspace_bytes, void *stream, int32_t *best_shape,
                                                  float *ms_per_step, int32_t ms_capacity) {
  tb_status status = check_batch_args("kpm_moments_batched_autotune", n_snap, n_rows, slice_ptr, col, val, precision,
                                      a, b, R, mode, workspace);
  if (status != TB_OK) return status;
  TB_REQUIRE(best_shape && reps >= 1 && reps <= 10000, "kpm_moments_batched_autotune: bad argument");
  TB_REQUIRE(ms_capacity >= 0 && (ms_capacity == 0 || ms_per_step), "kpm_moments_batched_autotune: bad ms buffer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  BatchLayout L;
  status = batch_layout(n_snap, n_rows, slice_ptr, true, st, &L);
  if (status != TB_OK) return status;
  FoldedBatch F;
  status = carve_folded(L, n_snap, precision == TB_F32 ? 4 : 8, workspace, workspace_bytes, &F);
  if (status != TB_OK) return status;
  status = upload_tables(L, n_snap, F, st);
  if (status == TB_OK) status = enqueue_fold(L, n_snap, slice_ptr, col, val, diag, precision, a, b, F, st);
  if (status != TB_OK) return status;
  int best = 0;
  // the segmented step, as the batch graph runs it
  const BatchDesc bd{F.tile, F.row0, F.rows, n_snap};
  const bool ok = precision == TB_F32
                      ? KpmEntry<float>::autotune(R, &status, L.n_pad, F.sp, F.col, F.val, F.diag, 1.0, 0.0, (int)mode,
                                                  (int)reps, F.run_ws, F.run_bytes, st, &best, ms_per_step,
                                                  ms_capacity, &bd)
                      : KpmEntry<double>::autotune(R, &status, L.n_pad, F.sp, F.col, F.val, F.diag, 1.0, 0.0,
                                                   (int)mode, (int)reps, F.run_ws, F.run_bytes, st, &best,
                                                   ms_per_step, ms_capacity, &bd);
  if (!ok) return fail(TB_ERR_INVALID_ARG, "kpm_moments_batched_autotune: unsupported R=%d", R);
  if (status != TB_OK) return status;
  *best_shape = best;
  return tb_kpm_set_shape(L.n_pad, R, precision, mode, best);
}

// ---------------------------------------------------------------------------
// Test hook for failure handling: the bounded wait that the pipelined step
// uses (an mbarrier phase), run on a phase that nothing completes, must give
// up after `polls` polls and report, leaving the context usable.
// ---------------------------------------------------------------------------
namespace gputb {
namespace {

__global__ void wait_probe_kernel(long long polls, int *__restrict__ status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);   // one arrival expected, none made
  __syncthreads();
  const bool ok = __syncthreads_and(mbar_wait_bounded(&bar, 0, polls)) != 0;
  if (threadIdx.x == 0) *status = ok ? 1 : 0;
}

}  // namespace
}  // namespace gputb

extern "C" tb_status tb_debug_wait_timeout(int64_t polls, void *workspace, size_t workspace_bytes, void *stream) {
  TB_REQUIRE(polls >= 1 && polls <= (int64_t(1) << 24), "tb_debug_wait_timeout: polls out of range");
  TB_REQUIRE(workspace && workspace_bytes >= 256, "tb_debug_wait_timeout: need 256 bytes of workspace");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int *status = static_cast<int *>(workspace);
  TB_CUDA(cudaMemsetAsync(status, 0, 256, st));
  wait_probe_kernel<<<1, kBlock, 0, st>>>((long long)polls, status);
  TB_CHECK_LAUNCH();
  int h = -1;
  TB_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  TB_CUDA(cudaStreamSynchronize(st));
  if (h == 0) return fail(TB_ERR_TIMEOUT, "tb_debug_wait_timeout: the mbarrier wait gave up after %lld polls",
                          (long long)polls);
  return TB_OK;
}
