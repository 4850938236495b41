// Error state and device queries of the C ABI.
#include <atomic>
#include <cstdarg>
#include <cstdio>

#include "common.cuh"

namespace gputb {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

tb_status fail(tb_status code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

tb_status cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
  set_error("CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(e),
            cudaGetErrorString(e), what, file, line);
  return TB_ERR_CUDA;
}

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long count) { g_launches.fetch_add(count, std::memory_order_relaxed); }

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 152;
  return n > 0 ? n : 152;
}

}  // namespace gputb

extern "C" int32_t tb_abi_version(void) { return GPUTB_ABI_VERSION; }
extern "C" const char *tb_last_error(void) { return gputb::g_err; }
extern "C" int64_t tb_launch_count(void) { return gputb::g_launches.load(); }

// Host <-> device copies of the C ABI (the boundary where host arrays enter
// and results leave): one cudaMemcpyAsync on `stream`; the copy to the host
// synchronises the stream so the data is there when the call returns.
extern "C" tb_status tb_copy_to_device(void *dst_device, const void *src_host, size_t bytes, void *stream) {
  TB_REQUIRE(bytes == 0 || (dst_device && src_host), "tb_copy_to_device: null pointer argument");
  if (bytes == 0) return TB_OK;
  TB_CUDA(cudaMemcpyAsync(dst_device, src_host, bytes, cudaMemcpyHostToDevice, static_cast<cudaStream_t>(stream)));
  return TB_OK;
}

extern "C" tb_status tb_copy_to_host(void *dst_host, const void *src_device, size_t bytes, void *stream) {
  TB_REQUIRE(bytes == 0 || (dst_host && src_device), "tb_copy_to_host: null pointer argument");
  if (bytes == 0) return TB_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TB_CUDA(cudaMemcpyAsync(dst_host, src_device, bytes, cudaMemcpyDeviceToHost, st));
  TB_CUDA(cudaStreamSynchronize(st));
  return TB_OK;
}
