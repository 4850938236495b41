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
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace gputb {
namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double phase_uniform(uint64_t seed, uint64_t r, uint64_t i) {
  const uint64_t z = splitmix64(seed ^ splitmix64((r << 32) + i));
  return static_cast<double>(z >> 11) * 0x1.0p-53;
}

// Each thread moves CPT complex numbers of one row: one 8-byte access
// (FP32, CPT = 1) or CPT*8/16 (FP32) / CPT (FP64) 16-byte accesses.
template <typename real, int CPT> struct Vec { using T = float4; static constexpr int kChunks = CPT / 2; };
template <> struct Vec<float, 1> { using T = float2; static constexpr int kChunks = 1; };
template <int CPT> struct Vec<double, CPT> { using T = double2; static constexpr int kChunks = CPT; };

// read-only cached load (neighbour gathers)
template <typename real, int CPT>
__device__ __forceinline__ void ld_gather(const real *p, real (&o)[2 * CPT]) {
  using V = typename Vec<real, CPT>::T;
#pragma unroll
  for (int k = 0; k < Vec<real, CPT>::kChunks; ++k) {
    V t = __ldg(reinterpret_cast<const V *>(p) + k);
    memcpy(o + k * (sizeof(V) / sizeof(real)), &t, sizeof(V));
  }
}
// streaming load / store (each element touched once per step)
template <typename real, int CPT>
__device__ __forceinline__ void ld_stream(const real *p, real (&o)[2 * CPT]) {
  using V = typename Vec<real, CPT>::T;
#pragma unroll
  for (int k = 0; k < Vec<real, CPT>::kChunks; ++k) {
    V t = __ldcs(reinterpret_cast<const V *>(p) + k);
    memcpy(o + k * (sizeof(V) / sizeof(real)), &t, sizeof(V));
  }
}
template <typename real, int CPT>
__device__ __forceinline__ void st_stream(real *p, const real (&v)[2 * CPT]) {
  using V = typename Vec<real, CPT>::T;
#pragma unroll
  for (int k = 0; k < Vec<real, CPT>::kChunks; ++k) {
    V t;
    memcpy(&t, v + k * (sizeof(V) / sizeof(real)), sizeof(V));
    __stcs(reinterpret_cast<V *>(p) + k, t);
  }
}

// Sum acc over all rows of the CTA for each of the R vectors and write the
// CTA's R partials.  Lanes that share `part` (lane mod TPR) hold the same
// vector components.
template <int R, int CPT>
__device__ __forceinline__ void cta_partial(double (&acc)[CPT], double *out) {
  constexpr int TPR = R / CPT;
  __shared__ double red[kWarps][R];
#pragma unroll
  for (int off = 16; off >= TPR; off >>= 1)
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < TPR)
#pragma unroll
    for (int c = 0; c < CPT; ++c) red[warp][lane * CPT + c] = acc[c];
  __syncthreads();
  if (threadIdx.x < R) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += red[w][threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// v0[i, r] = exp(2 pi i u(seed, r, i)); partial of mu_0 = Re <v0|v0>.
template <typename real, int R, int CPT>
__global__ void __launch_bounds__(kBlock) random_phase_kernel(int64_t n, uint64_t seed, real *__restrict__ v0,
                                                              double *__restrict__ partial) {
  constexpr int TPR = R / CPT;
  constexpr int RPB = kBlock / TPR;
  const int part = threadIdx.x % TPR;
  double acc[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) acc[c] = 0.0;
  for (int64_t row0 = (int64_t)blockIdx.x * RPB; row0 < n; row0 += (int64_t)gridDim.x * RPB) {
    const int64_t i = row0 + threadIdx.x / TPR;
    if (i < n) {
      real v[2 * CPT];
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int r = part * CPT + c;
        const double phi = 2.0 * M_PI * phase_uniform(seed, (uint64_t)r, (uint64_t)i);
        double s, co;
        sincos(phi, &s, &co);
        v[2 * c] = static_cast<real>(co);
        v[2 * c + 1] = static_cast<real>(s);
        acc[c] += (double)v[2 * c] * (double)v[2 * c] + (double)v[2 * c + 1] * (double)v[2 * c + 1];
      }
      st_stream<real, CPT>(v0 + (i * R + part * CPT) * 2, v);
    }
  }
  cta_partial<R, CPT>(acc, partial + (int64_t)blockIdx.x * R);
}

// One Chebyshev step over all rows:
//   out = alpha * (sum_s val x[col] + (diag_i - shift) x_i) - (FIRST ? 0 : prev)
// and the CTA partials of Re(conj(v0) out).  `prev` may alias `out`.
//
// The kernel is bound by HBM latency as much as by bandwidth: each row's
// gathers depend on its column loads, which depend on the slice offset.  So
// a row with at most kFastW slots issues all of its column and value loads
// first (predicated, fully unrolled), then all of its neighbour gathers,
// with the row's own v_{n-1} and v0 loads hoisted above them; wider rows take
// a plain loop.
constexpr int kFastW = 16;

template <typename real, typename valT, int R, int CPT, bool FIRST>
__global__ void __launch_bounds__(kBlock, (2 * CPT * sizeof(real) >= 32) ? 2 : 3) cheb_step_kernel(
    int64_t n, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ col,
    const valT *__restrict__ val, const valT *__restrict__ diag, const real *__restrict__ x,
    const real *prev, const real *__restrict__ v0, real *out, double *__restrict__ partial, real alpha,
    real shift) {
  constexpr int TPR = R / CPT;
  constexpr int RPB = kBlock / TPR;
  const int part = threadIdx.x % TPR;
  double acc[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) acc[c] = 0.0;
  for (int64_t row0 = (int64_t)blockIdx.x * RPB; row0 < n; row0 += (int64_t)gridDim.x * RPB) {
    const int64_t i = row0 + threadIdx.x / TPR;
    if (i < n) {
      const int64_t off = (i * R + part * CPT) * 2;
      real p[2 * CPT], z[2 * CPT];
      if (!FIRST) ld_stream<real, CPT>(prev + off, p);
      ld_stream<real, CPT>(v0 + off, z);
      const int64_t sb = __ldg(slice_ptr + (i >> 5));
      const int w = static_cast<int>((__ldg(slice_ptr + (i >> 5) + 1) - sb) >> 5);
      const int64_t e0 = sb + (i & 31);
      real y[2 * CPT];
#pragma unroll
      for (int c = 0; c < 2 * CPT; ++c) y[c] = real(0);
      if (w <= kFastW) {
        int32_t j[kFastW];
        real h[kFastW];
#pragma unroll
        for (int s = 0; s < kFastW; ++s) {
          if (s < w) {
            j[s] = __ldcs(col + e0 + 32 * s);
            h[s] = static_cast<real>(__ldcs(val + e0 + 32 * s));
          }
        }
#pragma unroll
        for (int s = 0; s < kFastW; ++s) {
          if (s < w) {
            real xv[2 * CPT];
            ld_gather<real, CPT>(x + ((int64_t)j[s] * R + part * CPT) * 2, xv);
#pragma unroll
            for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(h[s], xv[c], y[c]);
          }
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
      const real d = (diag ? static_cast<real>(__ldg(diag + i)) : real(0)) - shift;
      {
        real xi[2 * CPT];
        ld_gather<real, CPT>(x + off, xi);
#pragma unroll
        for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(d, xi[c], y[c]);
      }
      real o[2 * CPT];
#pragma unroll
      for (int c = 0; c < 2 * CPT; ++c) o[c] = FIRST ? alpha * y[c] : fma(alpha, y[c], -p[c]);
      st_stream<real, CPT>(out + off, o);
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        // Re(conj(v0) * o) = z.re o.re + z.im o.im, summed in FP64
        if (sizeof(real) == 4)
          acc[c] += (double)fmaf((float)z[2 * c], (float)o[2 * c], (float)z[2 * c + 1] * (float)o[2 * c + 1]);
        else
          acc[c] = fma((double)z[2 * c], (double)o[2 * c], fma((double)z[2 * c + 1], (double)o[2 * c + 1], acc[c]));
      }
    }
  }
  cta_partial<R, CPT>(acc, partial + (int64_t)blockIdx.x * R);
}

// mu_r[r, m] = (sum over CTAs in index order of partial[m, cta, r]) / n;
// flags[0] |= 1 if |mu| > 1 + 1e-6, |= 2 if not finite.
__global__ void moment_reduce_kernel(const double *__restrict__ partial, int grid, int R, int M, double inv_n,
                                     double *__restrict__ mu_r, int *__restrict__ flags) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)M * R) return;
  const int m = static_cast<int>(t / R), r = static_cast<int>(t % R);
  const double *p = partial + (int64_t)m * grid * R + r;
  double s = 0.0;
  for (int c = 0; c < grid; ++c) s += p[(int64_t)c * R];
  const double mu = s * inv_n;
  mu_r[(int64_t)r * M + m] = mu;
  if (!isfinite(mu)) atomicOr(flags, 2);
  else if (fabs(mu) > 1.0 + 1e-6) atomicOr(flags, 1);
}

template <typename real, typename valT, int R>
struct KpmRunner {
  // complex numbers per thread, chosen by measurement on GB300 (10M-atom
  // graphene): FP32 R = 4 -> 4 (two 16-byte accesses), other R >= 2 -> 2
  // (one 16-byte access), R = 1 -> 1; FP64 2 when R >= 2, else 1
  static constexpr int CPT = sizeof(real) == 4 ? (R == 4 ? 4 : (R >= 2 ? 2 : 1)) : (R >= 2 ? 2 : 1);
  static constexpr int TPR = R / CPT;
  static constexpr int RPB = kBlock / TPR;

  static int grid_for(int64_t n) {
    static int per_sm = 0;
    if (per_sm == 0) {
      int b = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cheb_step_kernel<real, valT, R, CPT, false>, kBlock, 0) !=
              cudaSuccess ||
          b <= 0)
        b = 4;
      per_sm = b;
    }
    const int64_t need = (n + RPB - 1) / RPB;
    const int64_t cap = (int64_t)per_sm * sm_count();
    return static_cast<int>(need < cap ? need : cap);
  }

  static size_t workspace(int64_t n, int M) {
    Carver cv(nullptr, 0);
    for (int k = 0; k < 3; ++k) cv.take<real>((size_t)n * R * 2);
    cv.take<double>((size_t)M * grid_for(n) * R);
    cv.take<int>(4);
    return cv.used + 256;
  }

  static tb_status run(int64_t n, const int64_t *slice_ptr, const int32_t *col, const valT *val, const valT *diag,
                       double a, double b, int M, uint64_t seed, double *mu_r, void *ws, size_t ws_bytes,
                       cudaStream_t st, double *step_ms) {
    const int grid = grid_for(n);
    Carver cv(ws, ws_bytes);
    real *v0 = cv.take<real>((size_t)n * R * 2);
    real *A = cv.take<real>((size_t)n * R * 2);
    real *B = cv.take<real>((size_t)n * R * 2);
    double *partial = cv.take<double>((size_t)M * grid * R);
    int *flags = cv.take<int>(4);
    if (!cv.ok()) return fail(TB_ERR_WORKSPACE, "kpm_moments: workspace too small (%zu < %zu)", ws_bytes, cv.used);
    TB_CUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
    random_phase_kernel<real, R, CPT><<<grid, kBlock, 0, st>>>(n, seed, v0, partial);
    TB_CHECK_LAUNCH();
    const real shift = static_cast<real>(b);
    const size_t pstride = (size_t)grid * R;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (step_ms) {
      TB_CUDA(cudaEventCreate(&ev[0]));
      TB_CUDA(cudaEventCreate(&ev[1]));
      TB_CUDA(cudaEventRecord(ev[0], st));
    }
    // v1 = H~ v0 -> A
    cheb_step_kernel<real, valT, R, CPT, true><<<grid, kBlock, 0, st>>>(
        n, slice_ptr, col, val, diag, v0, nullptr, v0, A, partial + pstride, static_cast<real>(1.0 / a), shift);
    TB_CHECK_LAUNCH();
    const real two_over_a = static_cast<real>(2.0 / a);
    for (int m = 2; m < M; ++m) {
      // v_m is written over v_{m-2}: m even -> B, m odd -> A; v_2 reads prev = v0
      real *out = (m & 1) ? A : B;
      const real *x = (m & 1) ? B : A;
      const real *prev = (m == 2) ? v0 : out;
      cheb_step_kernel<real, valT, R, CPT, false><<<grid, kBlock, 0, st>>>(
          n, slice_ptr, col, val, diag, x, prev, v0, out, partial + (size_t)m * pstride, two_over_a, shift);
      TB_CHECK_LAUNCH();
    }
    if (step_ms) TB_CUDA(cudaEventRecord(ev[1], st));
    const int total = M * R;
    moment_reduce_kernel<<<(total + 255) / 256, 256, 0, st>>>(partial, grid, R, M, 1.0 / (double)n, mu_r, flags);
    TB_CHECK_LAUNCH();
    int hflags[4] = {0, 0, 0, 0};
    TB_CUDA(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
    TB_CUDA(cudaStreamSynchronize(st));
    if (step_ms) {
      float ms = 0.f;
      TB_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
      *step_ms = ms;
      cudaEventDestroy(ev[0]);
      cudaEventDestroy(ev[1]);
    }
    if (hflags[0] & 2) return fail(TB_ERR_NOT_FINITE, "kpm_moments: non-finite moment");
    if (hflags[0] & 1)
      return fail(TB_ERR_BOUNDS, "kpm_moments: |mu_n| > 1 + 1e-6; the spectrum is not inside [b - a, b + a]");
    return TB_OK;
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

template <typename real, typename valT, int R>
struct WsOp {
  static tb_status apply(int64_t n, int M, size_t *out) {
    *out = KpmRunner<real, valT, R>::workspace(n, M);
    return TB_OK;
  }
};

template <typename real, typename valT, int R>
struct RunOp {
  static tb_status apply(int64_t n, const int64_t *sp, const int32_t *col, const void *val, const void *diag,
                         double a, double b, int M, uint64_t seed, double *mu, void *ws, size_t wsb,
                         cudaStream_t st, double *step_ms) {
    return KpmRunner<real, valT, R>::run(n, sp, col, static_cast<const valT *>(val),
                                         static_cast<const valT *>(diag), a, b, M, seed, mu, ws, wsb, st, step_ms);
  }
};

}  // namespace
}  // namespace gputb

using namespace gputb;

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
                                 uint64_t seed, double *mu_r, void *workspace, size_t workspace_bytes,
                                 void *stream, double *step_ms) {
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
                                                         seed, mu_r, workspace, workspace_bytes, st, step_ms)
                : KpmDispatch<double, double>::call<RunOp>(R, status, n, slice_ptr, col, val, diag, a, b, (int)M,
                                                           seed, mu_r, workspace, workspace_bytes, st, step_ms);
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
                                                         seed, mu_r, scratch, kNoAllocScratchBytes, st, nullptr)
                : KpmDispatch<double, double>::call<RunOp>(R, status, n, slice_ptr, col, val, diag, a, b, (int)M,
                                                           seed, mu_r, scratch, kNoAllocScratchBytes, st, nullptr);
  if (!ok) return fail(TB_ERR_INVALID_ARG, "kpm_moments_noalloc: unsupported R=%d", R);
  return status;
}
