// Shared host/device helpers of the CUDA library (error state, launch
// geometry, vector load/store).  Not shared with the oracle.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#include "gputb.h"

namespace gputb {

// thread-local message for tb_last_error()
void set_error(const char *fmt, ...);
tb_status fail(tb_status code, const char *fmt, ...);
tb_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);
int sm_count();
// process-wide count of kernel launches issued by the library (a graph
// launch adds the kernels it holds)
void note_launch();
void note_launches(long long count);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// carve 256-byte aligned sub-buffers out of a caller workspace
struct Carver {
  char *base;
  size_t cap;
  size_t used = 0;
  Carver(void *p, size_t c) : base(static_cast<char *>(p)), cap(c) {}
  template <typename T>
  T *take(size_t count) {
    used = align_up(used, 256);
    T *p = reinterpret_cast<T *>(base ? base + used : nullptr);
    used += count * sizeof(T);
    return p;
  }
  bool ok() const { return used <= cap; }
};

// Exclusive scan of int64 values (in may equal out); total (device) receives
// the sum.  Workspace from scan_workspace_bytes(n).  (scan.cu)
size_t scan_workspace_bytes(int64_t n);
tb_status exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total, void *ws,
                             cudaStream_t st);

}  // namespace gputb

#define TB_CUDA(call)                                                         \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) return gputb::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define TB_CHECK_LAUNCH()       \
  do {                          \
    gputb::note_launch();       \
    TB_CUDA(cudaGetLastError()); \
  } while (0)

#define TB_REQUIRE(cond, ...)                                                  \
  do {                                                                        \
    if (!(cond)) return gputb::fail(TB_ERR_INVALID_ARG, __VA_ARGS__);         \
  } while (0)
