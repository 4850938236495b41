// Multi-level exclusive prefix sum of int64 values (cell-list offsets and
// SELL-32 slice offsets).  Each CTA scans 1024 values with warp shuffles;
// CTA totals are scanned recursively and added back.
#include "geometry.cuh"

namespace gputb {
namespace {

constexpr int kScanBlock = 256;
constexpr int kPerThread = 4;
constexpr int kTile = kScanBlock * kPerThread;

__global__ void scan_tile_kernel(const int64_t *__restrict__ in, int64_t *__restrict__ out, int64_t n,
                                 int64_t *__restrict__ tile_sums) {
  __shared__ int64_t warp_sums[kScanBlock / 32];
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kPerThread;
  int64_t v[kPerThread];
  int64_t local = 0;
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    local += v[k];
  }
  // inclusive warp scan of per-thread totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t incl = local;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int64_t t = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += t;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < kScanBlock / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += t;
    }
    if (lane < kScanBlock / 32) warp_sums[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  int64_t run = incl - local + (warp > 0 ? warp_sums[warp - 1] : 0);
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == kScanBlock - 1) tile_sums[blockIdx.x] = run;  // last thread's run = tile total
}

__global__ void add_offsets_kernel(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ offs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += offs[i / kTile];
}

__global__ void copy_total_kernel(const int64_t *tile_sums, int64_t *total) { *total = tile_sums[0]; }

int64_t tiles(int64_t n) { return (n + kTile - 1) / kTile; }

}  // namespace

size_t scan_workspace_bytes(int64_t n) {
  size_t bytes = 0;
  int64_t m = n;
  do {
    m = tiles(m);
    bytes += align_up((size_t)m * sizeof(int64_t), 256);
  } while (m > 1);
  return bytes + 256;
}

tb_status exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total, void *ws,
                             cudaStream_t st) {
  if (n <= 0) {
    TB_CUDA(cudaMemsetAsync(total, 0, sizeof(int64_t), st));
    return TB_OK;
  }
  const int64_t t = tiles(n);
  int64_t *sums = static_cast<int64_t *>(ws);
  scan_tile_kernel<<<(unsigned)t, kScanBlock, 0, st>>>(in, out, n, sums);
  TB_CHECK_LAUNCH();
  if (t == 1) {
    copy_total_kernel<<<1, 1, 0, st>>>(sums, total);
    TB_CHECK_LAUNCH();
    return TB_OK;
  }
  char *next = static_cast<char *>(ws) + align_up((size_t)t * sizeof(int64_t), 256);
  tb_status s = exclusive_scan_i64(sums, sums, t, total, next, st);
  if (s != TB_OK) return s;
  add_offsets_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, sums);
  TB_CHECK_LAUNCH();
  return TB_OK;
}

}  // namespace gputb
