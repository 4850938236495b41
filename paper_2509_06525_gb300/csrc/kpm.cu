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

// acc + Re(conj(a) b) for complex a = (ar, ai), b = (br, bi): FP32 products
// summed into the FP64 accumulator (FP64 arithmetic for FP64 vectors)
template <typename real>
__device__ __forceinline__ double dot_acc(real ar, real ai, real br, real bi, double acc) {
  if (sizeof(real) == 4) return acc + (double)fmaf((float)ar, (float)br, (float)ai * (float)bi);
  return fma((double)ar, (double)br, fma((double)ai, (double)bi, acc));
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

template <typename real, typename valT, int R, int CPT, bool FIRST, bool DBL>
__global__ void __launch_bounds__(kBlock, (2 * CPT * sizeof(real) >= 32) ? 2 : 3) cheb_step_kernel(
    int64_t n, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ col,
    const valT *__restrict__ val, const valT *__restrict__ diag, const real *__restrict__ x,
    const real *prev, const real *__restrict__ v0, real *out, double *__restrict__ partial, real alpha,
    real shift) {
  constexpr int TPR = R / CPT;
  constexpr int RPB = kBlock / TPR;
  const int part = threadIdx.x % TPR;
  double acc[CPT], acc2[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) acc[c] = acc2[c] = 0.0;
  for (int64_t row0 = (int64_t)blockIdx.x * RPB; row0 < n; row0 += (int64_t)gridDim.x * RPB) {
    const int64_t i = row0 + threadIdx.x / TPR;
    if (i < n) {
      const int64_t off = (i * R + part * CPT) * 2;
      real p[2 * CPT], z[2 * CPT];
      if (!FIRST) ld_stream<real, CPT>(prev + off, p);
      if (!DBL) ld_stream<real, CPT>(v0 + off, z);
      const real d = (diag ? static_cast<real>(__ldg(diag + i)) : real(0)) - shift;
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
      real xi[2 * CPT];
      ld_gather<real, CPT>(x + off, xi);
#pragma unroll
      for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(d, xi[c], y[c]);
      real o[2 * CPT];
#pragma unroll
      for (int c = 0; c < 2 * CPT; ++c) o[c] = FIRST ? alpha * y[c] : fma(alpha, y[c], -p[c]);
      st_stream<real, CPT>(out + off, o);
      if (DBL) {
        // <v_n|v_n> and Re <v_n|v_{n+1}> for the doubling identities
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          acc[c] = dot_acc<real>(xi[2 * c], xi[2 * c + 1], xi[2 * c], xi[2 * c + 1], acc[c]);
          acc2[c] = dot_acc<real>(xi[2 * c], xi[2 * c + 1], o[2 * c], o[2 * c + 1], acc2[c]);
        }
      } else {
        // Re(conj(v0) * o) = z.re o.re + z.im o.im
#pragma unroll
        for (int c = 0; c < CPT; ++c) acc[c] = dot_acc<real>(z[2 * c], z[2 * c + 1], o[2 * c], o[2 * c + 1], acc[c]);
      }
    }
  }
  cta_partial<R, CPT>(acc, partial + (int64_t)blockIdx.x * R);
  if (DBL) {
    __syncthreads();
    cta_partial<R, CPT>(acc2, partial + (int64_t)gridDim.x * R + (int64_t)blockIdx.x * R);
  }
}

// ---------------------------------------------------------------------------
// Pipelined variant: the streamed operands of a tile of TR rows -- the tile's
// SELL slices of col and val (contiguous), and its rows of v_{n-1} and v0 --
// are moved by one elected thread with cp.async.bulk into a kStages-deep
// shared-memory ring whose stages complete on mbarriers (transaction
// counts).  All warps compute on one stage while the next ones are in
// flight, and the neighbour gathers take their indices from shared memory,
// so a row's gathers are issued without waiting for its column loads.  A
// tile whose slices are wider than kFastW falls back to direct loads of col
// and val.  Every wait is bounded: on timeout the CTA drains its own copies
// (bounded again), raises flags[0] |= 4 and returns.
// ---------------------------------------------------------------------------
constexpr int kStages = 3;
constexpr long long kWaitPolls = 1ll << 21;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  for (long long k = 0; k < kWaitPolls; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

template <typename real, typename valT, int R, int CPT>
struct BulkGeom {
  static constexpr int TPR = R / CPT;
  static constexpr int TR = kBlock / TPR;                       // rows per tile
  static constexpr int kEl = TR * kFastW;                       // SELL elements per stage
  static constexpr size_t kColBytes = kEl * sizeof(int32_t);
  static constexpr size_t kValBytes = kEl * sizeof(valT);
  static constexpr size_t kVecBytes = (size_t)TR * R * 2 * sizeof(real);
  static constexpr size_t kStageBytes = kColBytes + kValBytes + 2 * kVecBytes;
  static constexpr size_t kSmem = 128 + kStages * kStageBytes;  // mbarriers first
  static constexpr bool kOk = TR % 32 == 0 && kSmem <= 200 * 1024;
};

template <typename real, typename valT, int R, int CPT, bool FIRST, bool DBL>
__global__ void __launch_bounds__(kBlock) cheb_step_bulk_kernel(
    int64_t n, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ col,
    const valT *__restrict__ val, const valT *__restrict__ diag, const real *__restrict__ x, const real *prev,
    const real *__restrict__ v0, real *out, double *__restrict__ partial, real alpha, real shift,
    int *__restrict__ flags) {
  using G = BulkGeom<real, valT, R, CPT>;
  constexpr int TPR = G::TPR, TR = G::TR;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smem);
  unsigned char *ring = smem + 128;
  auto s_col = [&](int st) { return reinterpret_cast<int32_t *>(ring + st * G::kStageBytes); };
  auto s_val = [&](int st) { return reinterpret_cast<valT *>(ring + st * G::kStageBytes + G::kColBytes); };
  auto s_prev = [&](int st) {
    return reinterpret_cast<real *>(ring + st * G::kStageBytes + G::kColBytes + G::kValBytes);
  };
  auto s_v0 = [&](int st) {
    return reinterpret_cast<real *>(ring + st * G::kStageBytes + G::kColBytes + G::kValBytes + G::kVecBytes);
  };
  const int64_t ntiles = (n + TR - 1) / TR;
  const int part = threadIdx.x % TPR;
  const int lr = threadIdx.x / TPR;

  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) mbar_init(full + st, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // producer: stream the operands of local tile number kk into its stage
  auto issue = [&](int64_t kk) {
    const int64_t tile = blockIdx.x + kk * gridDim.x;
    const int st = static_cast<int>(kk % kStages);
    const int64_t r0 = tile * TR;
    const int64_t k0 = r0 >> 5;
    const int64_t k1 = min((r0 + TR + 31) >> 5, (n + 31) >> 5);
    const int64_t e0 = slice_ptr[k0], e1 = slice_ptr[k1];
    const bool bulk = (e1 - e0) <= G::kEl;
    const uint32_t ebytes = bulk ? static_cast<uint32_t>(e1 - e0) : 0u;
    uint32_t tx = static_cast<uint32_t>(G::kVecBytes) * ((FIRST ? 0u : 1u) + (DBL ? 0u : 1u));
    if (bulk) tx += ebytes * static_cast<uint32_t>(sizeof(int32_t) + sizeof(valT));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(full + st, tx);
    if (bulk && ebytes > 0) {
      bulk_g2s(s_col(st), col + e0, ebytes * sizeof(int32_t), full + st);
      bulk_g2s(s_val(st), val + e0, ebytes * sizeof(valT), full + st);
    }
    const size_t voff = (size_t)r0 * R * 2;
    if (!FIRST) bulk_g2s(s_prev(st), prev + voff, static_cast<uint32_t>(G::kVecBytes), full + st);
    if (!DBL) bulk_g2s(s_v0(st), v0 + voff, static_cast<uint32_t>(G::kVecBytes), full + st);
  };

  const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  int64_t issued = 0;
  if (threadIdx.x == 0)
    for (; issued < my_tiles && issued < kStages; ++issued) issue(issued);

  double acc[CPT], acc2[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) acc[c] = acc2[c] = 0.0;
  bool ok = true;
  int64_t kk = 0;
  for (; kk < my_tiles; ++kk) {
    const int st = static_cast<int>(kk % kStages);
    const uint32_t parity = static_cast<uint32_t>((kk / kStages) & 1);
    ok = __syncthreads_and(mbar_wait_bounded(full + st, parity)) != 0;
    if (!ok) break;
    const int64_t tile = blockIdx.x + kk * gridDim.x;
    const int64_t r0 = tile * TR;
    const int64_t i = r0 + lr;
    if (i < n) {
      const int64_t k0 = r0 >> 5;
      const int64_t k1 = min((r0 + TR + 31) >> 5, (n + 31) >> 5);
      const int64_t e0 = __ldg(slice_ptr + k0);
      const bool bulk = (__ldg(slice_ptr + k1) - e0) <= G::kEl;
      const int loff = (lr * R + part * CPT) * 2;
      real p[2 * CPT], z[2 * CPT];
      if (!FIRST) memcpy(p, s_prev(st) + loff, sizeof(p));
      if (!DBL) memcpy(z, s_v0(st) + loff, sizeof(z));
      const real d = (diag ? static_cast<real>(__ldg(diag + i)) : real(0)) - shift;
      const int64_t sb = __ldg(slice_ptr + (i >> 5));
      const int w = static_cast<int>((__ldg(slice_ptr + (i >> 5) + 1) - sb) >> 5);
      real y[2 * CPT];
#pragma unroll
      for (int c = 0; c < 2 * CPT; ++c) y[c] = real(0);
      if (bulk) {
        const int32_t *cs = s_col(st) + (sb - e0) + (i & 31);
        const valT *vs = s_val(st) + (sb - e0) + (i & 31);
#pragma unroll
        for (int s = 0; s < kFastW; ++s) {
          if (s < w) {
            real xv[2 * CPT];
            const real h = static_cast<real>(vs[32 * s]);
            ld_gather<real, CPT>(x + ((int64_t)cs[32 * s] * R + part * CPT) * 2, xv);
#pragma unroll
            for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(h, xv[c], y[c]);
          }
        }
      } else {
        int64_t e = sb + (i & 31);
        for (int s = 0; s < w; ++s, e += 32) {
          const int32_t jj = __ldcs(col + e);
          const real hh = static_cast<real>(__ldcs(val + e));
          real xv[2 * CPT];
          ld_gather<real, CPT>(x + ((int64_t)jj * R + part * CPT) * 2, xv);
#pragma unroll
          for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(hh, xv[c], y[c]);
        }
      }
      const int64_t off = (i * R + part * CPT) * 2;
      real xi[2 * CPT];
      ld_gather<real, CPT>(x + off, xi);
#pragma unroll
      for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(d, xi[c], y[c]);
      real o[2 * CPT];
#pragma unroll
      for (int c = 0; c < 2 * CPT; ++c) o[c] = FIRST ? alpha * y[c] : fma(alpha, y[c], -p[c]);
      st_stream<real, CPT>(out + off, o);
      if (DBL) {
        // <v_n|v_n> and Re <v_n|v_{n+1}> for the doubling identities
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          acc[c] = dot_acc<real>(xi[2 * c], xi[2 * c + 1], xi[2 * c], xi[2 * c + 1], acc[c]);
          acc2[c] = dot_acc<real>(xi[2 * c], xi[2 * c + 1], o[2 * c], o[2 * c + 1], acc2[c]);
        }
      } else {
        // Re(conj(v0) * o) = z.re o.re + z.im o.im
#pragma unroll
        for (int c = 0; c < CPT; ++c) acc[c] = dot_acc<real>(z[2 * c], z[2 * c + 1], o[2 * c], o[2 * c + 1], acc[c]);
      }
    }
    __syncthreads();  // every thread is done with this stage
    if (threadIdx.x == 0 && issued < my_tiles) issue(issued++);
  }
  if (!ok) {
    // drain this CTA's own copies still in flight, bounded, then report
    if (threadIdx.x == 0) {
      atomicOr(flags, 4);
      for (int64_t q = kk; q < issued; ++q)
        mbar_wait_bounded(full + q % kStages, static_cast<uint32_t>((q / kStages) & 1));
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[c] = acc2[c] = 0.0;
  }
  cta_partial<R, CPT>(acc, partial + (int64_t)blockIdx.x * R);
  if (DBL) {
    __syncthreads();
    cta_partial<R, CPT>(acc2, partial + (int64_t)gridDim.x * R + (int64_t)blockIdx.x * R);
  }
}

// mu_r[r, m] = (sum over CTAs in index order of partial[m, cta, r]) / n;
// flags[0] |= 1 if |mu| > 1 + 1e-6, |= 2 if not finite.
__device__ __forceinline__ double slot_sum(const double *__restrict__ partial, int grid, int R, int m, int r) {
  const double *p = partial + (int64_t)m * grid * R + r;
  double s = 0.0;
  for (int c = 0; c < grid; ++c) s += p[(int64_t)c * R];
  return s;
}

// direct mode: mu_m = S_m / n with S_m = sum_i Re conj(v0) v_m;
// doubling mode: S_0, S_1 as above, S_2k = sum |v_k|^2, S_2k+1 = sum Re conj(v_k) v_k+1,
// and mu_m = 2 S_m / n - mu_(m mod 2) for m >= 2 (Weisse et al. 2006)
__global__ void moment_reduce_kernel(const double *__restrict__ partial, int grid, int R, int M, double inv_n,
                                     int doubling, double *__restrict__ mu_r, int *__restrict__ flags) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)M * R) return;
  const int m = static_cast<int>(t / R), r = static_cast<int>(t % R);
  double mu = slot_sum(partial, grid, R, m, r) * inv_n;
  if (doubling && m >= 2) mu = 2.0 * mu - slot_sum(partial, grid, R, m & 1, r) * inv_n;
  mu_r[(int64_t)r * M + m] = mu;
  if (!isfinite(mu)) atomicOr(flags, 2);
  else if (fabs(mu) > 1.0 + 1e-6) atomicOr(flags, 1);
}

// kernel variant for the Chebyshev step: 0 = choose automatically,
// 1 = direct loads, 2 = bulk-copy pipeline (set with tb_kpm_set_variant)
int g_kpm_variant = 0;

template <typename real, typename valT, int R>
struct KpmRunner {
  // complex numbers per thread, chosen by measurement on GB300 (10M-atom
  // graphene): FP32 R = 4 -> 4 (two 16-byte accesses), other R >= 2 -> 2
  // (one 16-byte access), R = 1 -> 1; FP64 2 when R >= 2, else 1
  static constexpr int CPT = sizeof(real) == 4 ? (R == 4 ? 4 : (R >= 2 ? 2 : 1)) : (R >= 2 ? 2 : 1);
  static constexpr int TPR = R / CPT;
  static constexpr int RPB = kBlock / TPR;
  using G = BulkGeom<real, valT, R, CPT>;
  static constexpr int64_t kRowPad = 256;   // vector blocks hold whole tiles

  // the pipeline wins where several threads share a row (R >= 8 in FP32 on
  // GB300, measured); with one thread per row the direct kernel is faster
  static bool use_bulk() {
    if (!G::kOk || g_kpm_variant == 1) return false;
    return g_kpm_variant == 2 || TPR >= 4;
  }

  static int grid_for(int64_t n) {
    static int per_sm_direct = 0, per_sm_bulk = 0;
    if (use_bulk()) {
      if (per_sm_bulk == 0) {
        int b = 0;
        cudaFuncSetAttribute(cheb_step_bulk_kernel<real, valT, R, CPT, false, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::kSmem);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cheb_step_bulk_kernel<real, valT, R, CPT, false, false>,
                                                          kBlock, G::kSmem) != cudaSuccess ||
            b <= 0)
          b = 1;
        per_sm_bulk = b;
      }
      const int64_t need = (n + G::TR - 1) / G::TR;
      const int64_t cap = (int64_t)per_sm_bulk * sm_count();
      return static_cast<int>(need < cap ? need : cap);
    }
    if (per_sm_direct == 0) {
      int b = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cheb_step_kernel<real, valT, R, CPT, false, false>, kBlock, 0) !=
              cudaSuccess ||
          b <= 0)
        b = 4;
      per_sm_direct = b;
    }
    const int64_t need = (n + RPB - 1) / RPB;
    const int64_t cap = (int64_t)per_sm_direct * sm_count();
    return static_cast<int>(need < cap ? need : cap);
  }

  static int64_t padded_rows(int64_t n) { return (n + kRowPad - 1) / kRowPad * kRowPad; }

  static size_t workspace(int64_t n, int M) {
    Carver cv(nullptr, 0);
    for (int k = 0; k < 3; ++k) cv.take<real>((size_t)padded_rows(n) * R * 2);
    cv.take<double>((size_t)(M + 1) * grid_for(n) * R);
    cv.take<int>(4);
    return cv.used + 256;
  }

  template <bool FIRST, bool DBL>
  static tb_status step(int grid, int64_t n, const int64_t *slice_ptr, const int32_t *col, const valT *val,
                        const valT *diag, const real *x, const real *prev, const real *v0, real *out,
                        double *partial, real alpha, real shift, int *flags, cudaStream_t st) {
    if (use_bulk()) {
      cudaFuncSetAttribute(cheb_step_bulk_kernel<real, valT, R, CPT, FIRST, DBL>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::kSmem);
      cheb_step_bulk_kernel<real, valT, R, CPT, FIRST, DBL><<<grid, kBlock, G::kSmem, st>>>(
          n, slice_ptr, col, val, diag, x, prev, v0, out, partial, alpha, shift, flags);
    } else {
      cheb_step_kernel<real, valT, R, CPT, FIRST, DBL><<<grid, kBlock, 0, st>>>(n, slice_ptr, col, val, diag, x,
                                                                               prev, v0, out, partial, alpha, shift);
    }
    TB_CHECK_LAUNCH();
    return TB_OK;
  }

  static tb_status run(int64_t n, const int64_t *slice_ptr, const int32_t *col, const valT *val, const valT *diag,
                       double a, double b, int M, uint64_t seed, int mode, double *mu_r, void *ws,
                       size_t ws_bytes, cudaStream_t st, double *step_ms) {
    const int grid = grid_for(n);
    const int64_t np = padded_rows(n);
    const bool dbl = mode == TB_KPM_DOUBLING;
    Carver cv(ws, ws_bytes);
    real *v0 = cv.take<real>((size_t)np * R * 2);
    real *A = cv.take<real>((size_t)np * R * 2);
    real *B = cv.take<real>((size_t)np * R * 2);
    double *partial = cv.take<double>((size_t)(M + 1) * grid * R);
    int *flags = cv.take<int>(4);
    if (!cv.ok()) return fail(TB_ERR_WORKSPACE, "kpm_moments: workspace too small (%zu < %zu)", ws_bytes, cv.used);
    if (use_bulk() && ((reinterpret_cast<uintptr_t>(col) | reinterpret_cast<uintptr_t>(val)) & 15))
      return fail(TB_ERR_INVALID_ARG, "kpm_moments: col and val must be 16-byte aligned");
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
    // v1 = H~ v0 -> A.  Direct mode: the step making v_m adds the partials of
    // mu_m; doubling mode: the step reading v_k adds those of S_2k and S_2k+1.
    const real inv_a = static_cast<real>(1.0 / a);
    tb_status s = dbl ? step<true, true>(grid, n, slice_ptr, col, val, diag, v0, nullptr, v0, A, partial, inv_a,
                                         shift, flags, st)
                      : step<true, false>(grid, n, slice_ptr, col, val, diag, v0, nullptr, v0, A,
                                          partial + pstride, inv_a, shift, flags, st);
    if (s != TB_OK) return s;
    const real two_over_a = static_cast<real>(2.0 / a);
    const int last = dbl ? (M - 1) / 2 + 1 : M - 1;   // index of the last vector computed
    for (int m = 2; m <= last; ++m) {
      // v_m is written over v_{m-2}: m even -> B, m odd -> A; v_2 reads prev = v0
      real *out = (m & 1) ? A : B;
      const real *x = (m & 1) ? B : A;
      const real *prev = (m == 2) ? v0 : out;
      s = dbl ? step<false, true>(grid, n, slice_ptr, col, val, diag, x, prev, v0, out,
                                  partial + (size_t)(2 * (m - 1)) * pstride, two_over_a, shift, flags, st)
              : step<false, false>(grid, n, slice_ptr, col, val, diag, x, prev, v0, out,
                                   partial + (size_t)m * pstride, two_over_a, shift, flags, st);
      if (s != TB_OK) return s;
    }
    if (step_ms) TB_CUDA(cudaEventRecord(ev[1], st));
    const int total = M * R;
    moment_reduce_kernel<<<(total + 255) / 256, 256, 0, st>>>(partial, grid, R, M, 1.0 / (double)n, dbl ? 1 : 0,
                                                              mu_r, flags);
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
    if (hflags[0] & 4) return fail(TB_ERR_TIMEOUT, "kpm_moments: a pipeline wait timed out");
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
                         double a, double b, int M, uint64_t seed, int mode, double *mu, void *ws, size_t wsb,
                         cudaStream_t st, double *step_ms) {
    return KpmRunner<real, valT, R>::run(n, sp, col, static_cast<const valT *>(val),
                                         static_cast<const valT *>(diag), a, b, M, seed, mode, mu, ws, wsb, st,
                                         step_ms);
  }
};

}  // namespace
}  // namespace gputb

using namespace gputb;

extern "C" tb_status tb_kpm_set_variant(int32_t variant) {
  TB_REQUIRE(variant >= 0 && variant <= 2, "tb_kpm_set_variant: variant must be 0, 1 or 2");
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
                                 uint64_t seed, int32_t mode, double *mu_r, void *workspace,
                                 size_t workspace_bytes, void *stream, double *step_ms) {
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
                                                         seed, (int)mode, mu_r, workspace, workspace_bytes, st,
                                                         step_ms)
                : KpmDispatch<double, double>::call<RunOp>(R, status, n, slice_ptr, col, val, diag, a, b, (int)M,
                                                           seed, (int)mode, mu_r, workspace, workspace_bytes, st,
                                                           step_ms);
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
                                                         seed, (int)TB_KPM_DIRECT, mu_r, scratch,
                                                         kNoAllocScratchBytes, st, nullptr)
                : KpmDispatch<double, double>::call<RunOp>(R, status, n, slice_ptr, col, val, diag, a, b, (int)M,
                                                           seed, (int)TB_KPM_DIRECT, mu_r, scratch,
                                                           kNoAllocScratchBytes, st, nullptr);
  if (!ok) return fail(TB_ERR_INVALID_ARG, "kpm_moments_noalloc: unsupported R=%d", R);
  return status;
}
