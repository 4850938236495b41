// Chebyshev-step machinery shared by the KPM moments (kpm_*.cu) and the VAC
// conductivity (lsqt.cu): the direct-load and bulk-copy-pipeline step
// kernels, templated on their launch shape; the table of candidate shapes
// per (precision, R) that the autotuner chooses from; the moment partial
// flush and the fixed-order moment reduction.  Everything below the kpmdev
// declarations has internal linkage in each translation unit that includes
// it.
#pragma once

#include <algorithm>
#include <type_traits>
#include <utility>

#include "kpm_band.cuh"
#include "kpm_common.cuh"

namespace gputb {
namespace kpmdev {
// Shape of the Chebyshev step chosen for a call (see kpm_shapes.cu): an
// explicitly forced shape, else the autotuned one for the size class of n,
// else 0 (the default shape of every candidate list).
int chosen_shape(int precision, int R, int mode, int64_t n);
}  // namespace kpmdev

namespace {
using namespace kpmdev;

// Batch description (device tables) for kpm_moments_batched: rows of
// snapshot s occupy [row0[s], row0[s] + padded) of the concatenated blocks,
// the first rows[s] of them real; tile_snap maps each 256-row tile to its
// snapshot.
struct BatchTables {
  const int32_t *tile_snap = nullptr;
  const int64_t *row0 = nullptr;
  const int64_t *rows = nullptr;
  int n_snap = 0;
};
constexpr int kBatchTile = 256;

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

// Write the CTA's partial sums as entry `idx` of the moment slot (and of the
// next slot for the doubling pair), then restart the accumulators.  Every
// thread of the CTA must call it.
template <typename real, int R, int CPT, bool DBL, typename Acc>
__device__ __forceinline__ void flush_partials(Acc (&acc)[CPT], Acc (&acc2)[CPT], double *partial, int64_t idx,
                                               int64_t slot_stride) {
  double sum[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) sum[c] = acc[c].value();
  cta_partial<R, CPT>(sum, partial + idx * R);
  __syncthreads();
  if (DBL) {
#pragma unroll
    for (int c = 0; c < CPT; ++c) sum[c] = acc2[c].value();
    cta_partial<R, CPT>(sum, partial + slot_stride + idx * R);
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < CPT; ++c) acc[c] = acc2[c] = Acc();
}

// The order in which a CTA visits the tiles (or row blocks): chunks of C
// consecutive tiles, the chunks dealt out grid-stride.  C = 1 is the plain
// grid-stride order of the single-matrix path.  C = 0 gives each CTA one
// contiguous span of about ntiles / grid tiles: the segmented (batched) mode
// takes it, so that a CTA's run within one snapshot ends only where the
// snapshot does (one reduction per snapshot the span meets).
constexpr int kSegChunk = 0;
template <int C>
struct TileWalk {
  int64_t ntiles, nchunks;
  __device__ __forceinline__ explicit TileWalk(int64_t nt) : ntiles(nt), nchunks((nt + C - 1) / C) {}
  // tiles this CTA visits (the last chunk may be short)
  __device__ __forceinline__ int64_t count() const {
    const int64_t b = blockIdx.x;
    if (b >= nchunks) return 0;
    const int64_t owned = (nchunks - 1 - b) / gridDim.x + 1;
    const bool last = (nchunks - 1 - b) % gridDim.x == 0;
    return owned * C - (last ? nchunks * C - ntiles : 0);
  }
  __device__ __forceinline__ int64_t tile(int64_t kk) const {
    return ((kk / C) * gridDim.x + blockIdx.x) * C + kk % C;
  }
};
template <>
struct TileWalk<0> {
  int64_t first, n;
  __device__ __forceinline__ explicit TileWalk(int64_t nt) {
    const int64_t per = (nt + gridDim.x - 1) / gridDim.x;
    first = min(nt, (int64_t)blockIdx.x * per);
    n = min(nt, first + per) - first;
  }
  __device__ __forceinline__ int64_t count() const { return n; }
  __device__ __forceinline__ int64_t tile(int64_t kk) const { return first + kk; }
};

// Segmented mode: block `blk` of the current run of RPB-row blocks has just
// been processed; `nxt` is this CTA's next block (-1 if none).  Every block
// of a run except its first gets zeros; when the next block lies in another
// snapshot (or there is none) the run's sums go into the entry of the run's
// first block.  Uniform across the CTA.
template <typename real, int R, int CPT, bool DBL, typename Acc>
__device__ __forceinline__ void segment_boundary(Acc (&acc)[CPT], Acc (&acc2)[CPT],
                                                 double *partial, int64_t slot_stride, const BatchTables &bt,
                                                 int64_t blk, int rpb, int64_t nxt, int64_t &run_head) {
  // snapshots start on kBatchTile-row boundaries: blocks inside one such
  // group share their snapshot, so only a group change needs the table
  const int64_t g_nxt = (nxt * rpb) / kBatchTile, g_blk = (blk * rpb) / kBatchTile;
  const bool ends = nxt < 0 || (g_nxt != g_blk && __ldg(bt.tile_snap + g_nxt) != __ldg(bt.tile_snap + g_blk));
  if (blk != run_head && threadIdx.x < R) {  // every block but the run's first holds zero
    partial[blk * R + threadIdx.x] = 0.0;
    if (DBL) partial[slot_stride + blk * R + threadIdx.x] = 0.0;
  }
  if (ends) {
    flush_partials<real, R, CPT, DBL>(acc, acc2, partial, run_head, slot_stride);
    run_head = nxt;
  }
}

// The row's product y = sum_s h_s x[j_s] (CPT complex numbers of the
// thread's share of the R vectors) with the slot loads issued first.
template <typename real, typename valT, int R, int CPT>
__device__ __forceinline__ void row_product_direct(const int32_t *__restrict__ col, const valT *__restrict__ val,
                                                   const real *__restrict__ x, int64_t e0, int w, int part,
                                                   real (&y)[2 * CPT]) {
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
}

// The row's tail shared by both kernels: the diagonal term, the output
// (stored with evict-first) and the dot accumulation.
template <typename real, int CPT, bool FIRST, bool DBL, typename Acc>
__device__ __forceinline__ void row_finish(real (&y)[2 * CPT], const real (&xi)[2 * CPT], const real (&p)[2 * CPT],
                                           const real (&z)[2 * CPT], real d, real alpha, real *out, Acc (&acc)[CPT],
                                           Acc (&acc2)[CPT]) {
#pragma unroll
  for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(d, xi[c], y[c]);
  real o[2 * CPT];
#pragma unroll
  for (int c = 0; c < 2 * CPT; ++c) o[c] = FIRST ? alpha * y[c] : fma(alpha, y[c], -p[c]);
  st_stream<real, CPT>(out, o);
  if (DBL) {
    // <v_n|v_n> and Re <v_n|v_{n+1}> for the doubling identities
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      acc[c].add(xi[2 * c], xi[2 * c + 1], xi[2 * c], xi[2 * c + 1]);
      acc2[c].add(xi[2 * c], xi[2 * c + 1], o[2 * c], o[2 * c + 1]);
    }
  } else {
    // Re(conj(v0) * o) = z.re o.re + z.im o.im
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[c].add(z[2 * c], z[2 * c + 1], o[2 * c], o[2 * c + 1]);
  }
}

template <typename real, typename valT, int R, int CPT, int MINB, bool FIRST, bool DBL, bool SEG>
__global__ void __launch_bounds__(kBlock, MINB) cheb_step_kernel(
    int64_t n, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ col,
    const valT *__restrict__ val, const valT *__restrict__ diag, const real *__restrict__ x,
    const real *prev, const real *__restrict__ v0, real *out, double *__restrict__ partial, real alpha,
    real shift, int64_t slot_stride, BatchTables bt) {
  constexpr int TPR = R / CPT;
  constexpr int RPB = kBlock / TPR;
  const int part = threadIdx.x % TPR;
  DotAcc<real> acc[CPT], acc2[CPT];
  // SEG (batched): the CTA's blocks (one contiguous span) form runs within
  // one snapshot, reduced where the snapshot changes; other blocks' entries
  // are 0
  const TileWalk<SEG ? kSegChunk : 1> walk((n + RPB - 1) / RPB);
  const int64_t my_blocks = walk.count();
  int64_t run_head = walk.tile(0);
  for (int64_t kb = 0; kb < my_blocks; ++kb) {
    const int64_t blk = walk.tile(kb);
    const int64_t row0 = blk * RPB;
    const int64_t i = row0 + threadIdx.x / TPR;
    if (i < n) {
      const int64_t off = (i * R + part * CPT) * 2;
      real p[2 * CPT], z[2 * CPT];
      if (!FIRST) ld_stream<real, CPT>(prev + off, p);
      if (!DBL) ld_stream<real, CPT>(v0 + off, z);
      const real d = (diag ? static_cast<real>(__ldg(diag + i)) : real(0)) - shift;
      const int64_t sb = __ldg(slice_ptr + (i >> 5));
      const int w = static_cast<int>((__ldg(slice_ptr + (i >> 5) + 1) - sb) >> 5);
      real y[2 * CPT];
#pragma unroll
      for (int c = 0; c < 2 * CPT; ++c) y[c] = real(0);
      row_product_direct<real, valT, R, CPT>(col, val, x, sb + (i & 31), w, part, y);
      real xi[2 * CPT];
      ld_gather<real, CPT>(x + off, xi);
      row_finish<real, CPT, FIRST, DBL>(y, xi, p, z, d, alpha, out + off, acc, acc2);
    }
    if (SEG)
      segment_boundary<real, R, CPT, DBL>(acc, acc2, partial, slot_stride, bt, blk, RPB,
                                          kb + 1 < my_blocks ? walk.tile(kb + 1) : -1, run_head);
  }
  if (!SEG) flush_partials<real, R, CPT, DBL>(acc, acc2, partial, blockIdx.x, slot_stride);
}

// ---------------------------------------------------------------------------
// Pipelined variant: the streamed operands of a tile of TR rows -- the tile's
// SELL slices of col and val (contiguous), and its rows of v_{n-1} and v0 --
// are moved by one elected thread with cp.async.bulk into a STAGES-deep
// shared-memory ring whose stages complete on mbarriers (transaction
// counts).  All warps compute on one stage while the next ones are in
// flight, and the neighbour gathers take their indices from shared memory,
// so a row's gathers are issued without waiting for its column loads.  A
// tile with more elements than a stage holds (TR x kFastW) falls back to
// direct loads of col and val; a slice wider than kFastW in a tile that fits
// loops over its slots in shared memory.  Every wait is bounded: on timeout the CTA drains its own copies
// (bounded again), raises flags[0] |= 4 and returns.
// ---------------------------------------------------------------------------
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
// the same test, letting the thread sleep up to `ns` nanoseconds for the
// phase (it wakes when the phase completes)
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
constexpr uint32_t kWaitSleepNs = 2000;
// at most `polls` tests (each may sleep up to kWaitSleepNs): a few seconds
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long polls = kWaitPolls) {
  if (polls > 0 && mbar_try_wait(bar, parity)) return true;
  for (long long k = 1; k < polls; ++k)
    if (mbar_try_wait_sleep(bar, parity, kWaitSleepNs)) return true;
  return false;
}

// NV: vector rows streamed per stage (v_{n-1}, and v0 unless in doubling mode)
template <typename real, typename valT, int R, int CPT, int STAGES, int NV = 2>
struct BulkGeom {
  static constexpr int TPR = R / CPT;
  static constexpr int TR = kBlock / TPR;                       // rows per tile
  static constexpr int kEl = TR * kFastW;                       // SELL elements per stage
  static constexpr size_t kColBytes = kEl * sizeof(int32_t);
  static constexpr size_t kValBytes = kEl * sizeof(valT);
  static constexpr size_t kVecBytes = (size_t)TR * R * 2 * sizeof(real);
  static constexpr size_t kStageBytes = kColBytes + kValBytes + NV * kVecBytes;
  static constexpr size_t kSmem = 128 + STAGES * kStageBytes;  // mbarriers first
  static constexpr bool kOk = TR % 32 == 0 && kSmem <= 200 * 1024 && STAGES >= 2 && STAGES <= 8;
};

// y += sum over the row's slots (from shared memory) of h_s x[j_s]
template <typename real, typename valT, int R, int CPT, int W>
__device__ __forceinline__ void row_product_smem(const int32_t *cs, const valT *vs, const real *__restrict__ xp,
                                                 int w, real (&y)[2 * CPT]) {
#pragma unroll
  for (int s = 0; s < W; ++s) {
    if (s < w) {
      real xv[2 * CPT];
      const real h = static_cast<real>(vs[32 * s]);
      ld_gather<real, CPT>(xp + (int64_t)cs[32 * s] * (R * 2), xv);
#pragma unroll
      for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(h, xv[c], y[c]);
    }
  }
}

// Option of the ring kernel (bit mask OPT, chosen per shape):
//   1  rows of slices at most 12 wide take a 12-slot unrolled body
template <typename real, typename valT, int R, int CPT, int STAGES, int MINB, int OPT, bool FIRST, bool DBL, bool SEG>
__global__ void __launch_bounds__(kBlock, MINB) cheb_step_bulk_kernel(
    int64_t n, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ col,
    const valT *__restrict__ val, const valT *__restrict__ diag, const real *__restrict__ x, const real *prev,
    const real *__restrict__ v0, real *out, double *__restrict__ partial, real alpha, real shift,
    int *__restrict__ flags, int64_t slot_stride, BatchTables bt) {
  using G = BulkGeom<real, valT, R, CPT, STAGES, DBL ? 1 : 2>;
  using Acc = DotAcc<real>;
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
  // tiles of this CTA: grid-stride (one contiguous span in SEG mode)
  const TileWalk<SEG ? kSegChunk : 1> walk(ntiles);   // this CTA's tiles, in order
  auto tile_of = [&](int64_t kk) { return walk.tile(kk); };

  if (threadIdx.x == 0) {
    for (int st = 0; st < STAGES; ++st) mbar_init(full + st, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // producer: stream the operands of local tile number kk into its stage
  auto issue = [&](int64_t kk) {
    const int64_t tile = tile_of(kk);
    const int st = static_cast<int>(kk % STAGES);
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

  const int64_t my_tiles = walk.count();
  int64_t run_head = tile_of(0);
  int64_t issued = 0;
  if (threadIdx.x == 0)
    for (; issued < my_tiles && issued < STAGES; ++issued) issue(issued);

  Acc acc[CPT], acc2[CPT];
  bool ok = true;
  int64_t kk = 0;
  for (; kk < my_tiles; ++kk) {
    const int st = static_cast<int>(kk % STAGES);
    const uint32_t parity = static_cast<uint32_t>((kk / STAGES) & 1);
    ok = __syncthreads_and(mbar_wait_bounded(full + st, parity)) != 0;
    if (!ok) break;
    const int64_t tile = tile_of(kk);
    const int64_t r0 = tile * TR;
    const int64_t i = r0 + lr;
    if (i < n) {
      const int64_t k0 = r0 >> 5;
      const int64_t k1 = min((r0 + TR + 31) >> 5, (n + 31) >> 5);
      const int64_t e0 = __ldg(slice_ptr + k0);
      const bool bulk = (__ldg(slice_ptr + k1) - e0) <= G::kEl;
      const int64_t sb = __ldg(slice_ptr + (i >> 5));
      const int w = static_cast<int>((__ldg(slice_ptr + (i >> 5) + 1) - sb) >> 5);
      const int loff = (lr * R + part * CPT) * 2;
      real p[2 * CPT], z[2 * CPT];
      if (!FIRST) memcpy(p, s_prev(st) + loff, sizeof(p));
      if (!DBL) memcpy(z, s_v0(st) + loff, sizeof(z));
      const real d = (diag ? static_cast<real>(__ldg(diag + i)) : real(0)) - shift;
      real y[2 * CPT];
#pragma unroll
      for (int c = 0; c < 2 * CPT; ++c) y[c] = real(0);
      if (bulk) {
        const int32_t *cs = s_col(st) + (sb - e0) + (i & 31);
        const valT *vs = s_val(st) + (sb - e0) + (i & 31);
        const real *xp = x + part * CPT * 2;
        if ((OPT & 1) && w <= 12) {
          row_product_smem<real, valT, R, CPT, 12>(cs, vs, xp, w, y);
        } else if (w <= kFastW) {
          row_product_smem<real, valT, R, CPT, kFastW>(cs, vs, xp, w, y);
        } else {
          // a slice wider than kFastW inside a tile that still fits the stage
#pragma unroll 1
          for (int s = 0; s < w; ++s) {
            real xv[2 * CPT];
            const real h = static_cast<real>(vs[32 * s]);
            ld_gather<real, CPT>(xp + (int64_t)cs[32 * s] * (R * 2), xv);
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
      row_finish<real, CPT, FIRST, DBL>(y, xi, p, z, d, alpha, out + off, acc, acc2);
    }
    if (SEG)
      segment_boundary<real, R, CPT, DBL>(acc, acc2, partial, slot_stride, bt, tile, TR,
                                          kk + 1 < my_tiles ? tile_of(kk + 1) : -1, run_head);
    __syncthreads();  // every thread is done with this stage
    if (threadIdx.x == 0 && issued < my_tiles) issue(issued++);
  }
  if (!ok) {
    // drain this CTA's own copies still in flight, bounded, then report
    if (threadIdx.x == 0) {
      atomicOr(flags, 4);
      for (int64_t q = kk; q < issued; ++q)
        mbar_wait_bounded(full + q % STAGES, static_cast<uint32_t>((q / STAGES) & 1));
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[c] = acc2[c] = Acc();
  }
  if (!SEG) flush_partials<real, R, CPT, DBL>(acc, acc2, partial, blockIdx.x, slot_stride);
}

// ---------------------------------------------------------------------------
// Second ring kernel: per tile of TR = RPT x (kBlock / TPR) rows the stage
// also holds the tile's slice offsets (written by warp 0 from slice_ptr) and
// its diagonal entries (bulk-copied with col and val), so that a consumer
// thread issues no global load but its neighbour gathers, its own row of x
// and (with STAGE_VEC = false) its streamed rows of v_{n-1} and v0.  Each
// thread takes RPT rows per tile, which spreads the per-tile waits and
// barriers over RPT rows.  Rows of slices at most 12 wide (graphene's 12
// neighbours within 3 A) take a 12-slot unrolled body.
// ---------------------------------------------------------------------------
template <typename real, typename valT, int R, int CPT, int STAGES, int RPT, bool STAGE_VEC, int NV>
struct Ring2Geom {
  static constexpr int TPR = R / CPT;
  static constexpr int TRW = kBlock / TPR;                      // rows per wave of the CTA
  static constexpr int TR = TRW * RPT;                          // rows per tile
  static constexpr int kSlices = TR / 32;
  static constexpr int kEl = TR * kFastW;                       // SELL elements per stage
  static constexpr size_t kHdrBytes = ((kSlices + 1) * 8 + 15) / 16 * 16;
  static constexpr size_t kColBytes = kEl * sizeof(int32_t);
  static constexpr size_t kValBytes = kEl * sizeof(valT);
  static constexpr size_t kDiagBytes = (TR * sizeof(valT) + 15) / 16 * 16;
  static constexpr size_t kVecBytes = (size_t)TR * R * 2 * sizeof(real);
  static constexpr size_t kStageBytes = kHdrBytes + kColBytes + kValBytes + kDiagBytes + (STAGE_VEC ? NV : 0) * kVecBytes;
  static constexpr size_t kSmem = 128 + STAGES * kStageBytes;
  static constexpr bool kOk = TRW % 32 == 0 && kSmem <= 200 * 1024 && STAGES >= 2 && STAGES <= 8 && kSlices + 1 <= 32;
};

template <typename real, typename valT, int R, int CPT, int STAGES, int MINB, int RPT, bool STAGE_VEC, bool FIRST,
          bool DBL, bool SEG>
__global__ void __launch_bounds__(kBlock, MINB) cheb_step_ring2_kernel(
    int64_t n, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ col,
    const valT *__restrict__ val, const valT *__restrict__ diag, const real *__restrict__ x, const real *prev,
    const real *__restrict__ v0, real *out, double *__restrict__ partial, real alpha, real shift,
    int *__restrict__ flags, int64_t slot_stride, BatchTables bt) {
  using G = Ring2Geom<real, valT, R, CPT, STAGES, RPT, STAGE_VEC, DBL ? 1 : 2>;
  constexpr int TPR = G::TPR, TRW = G::TRW, TR = G::TR;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smem);
  unsigned char *ring = smem + 128;
  auto s_hdr = [&](int st) { return reinterpret_cast<int64_t *>(ring + st * G::kStageBytes); };
  auto s_col = [&](int st) { return reinterpret_cast<int32_t *>(ring + st * G::kStageBytes + G::kHdrBytes); };
  auto s_val = [&](int st) {
    return reinterpret_cast<valT *>(ring + st * G::kStageBytes + G::kHdrBytes + G::kColBytes);
  };
  auto s_diag = [&](int st) {
    return reinterpret_cast<valT *>(ring + st * G::kStageBytes + G::kHdrBytes + G::kColBytes + G::kValBytes);
  };
  auto s_vec = [&](int st, int q) {
    return reinterpret_cast<real *>(ring + st * G::kStageBytes + G::kHdrBytes + G::kColBytes + G::kValBytes +
                                    G::kDiagBytes + q * G::kVecBytes);
  };
  const int64_t ntiles = (n + TR - 1) / TR;
  const int64_t n_slices = (n + 31) >> 5;
  const int part = threadIdx.x % TPR;
  const int lr0 = threadIdx.x / TPR;
  const TileWalk<SEG ? kSegChunk : 1> walk(ntiles);   // this CTA's tiles, in order
  auto tile_of = [&](int64_t kk) { return walk.tile(kk); };
  const real *xp = x + part * CPT * 2;   // this thread's components of every row of x

  if (threadIdx.x == 0) {
    for (int st = 0; st < STAGES; ++st) mbar_init(full + st, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // producer (warp 0): the tile's slice offsets into the header, then the
  // bulk copies of col, val, diag (whole tiles) and the staged vector rows
  auto issue = [&](int64_t kk) {
    const int lane = threadIdx.x & 31;
    const int64_t tile = tile_of(kk);
    const int st = static_cast<int>(kk % STAGES);
    const int64_t r0 = tile * TR;
    const int64_t k0 = r0 >> 5;
    const int64_t k1 = min(k0 + G::kSlices, n_slices);
    int64_t off = 0;
    if (lane <= G::kSlices) {
      off = slice_ptr[min(k0 + lane, k1)];
      s_hdr(st)[lane] = off;
    }
    const int64_t e0 = __shfl_sync(0xffffffffu, off, 0);
    const int64_t e1 = __shfl_sync(0xffffffffu, off, G::kSlices);
    __syncwarp();
    if (lane == 0) {
      const bool bulk = (e1 - e0) <= G::kEl;
      const bool whole = r0 + TR <= n;
      const uint32_t ebytes = bulk ? static_cast<uint32_t>(e1 - e0) : 0u;
      uint32_t tx = 0;
      if (bulk) tx += ebytes * static_cast<uint32_t>(sizeof(int32_t) + sizeof(valT));
      if (diag && whole) tx += TR * sizeof(valT);
      if (STAGE_VEC) tx += static_cast<uint32_t>(G::kVecBytes) * ((FIRST ? 0u : 1u) + (DBL ? 0u : 1u));
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(full + st, tx);
      if (bulk && ebytes > 0) {
        bulk_g2s(s_col(st), col + e0, ebytes * sizeof(int32_t), full + st);
        bulk_g2s(s_val(st), val + e0, ebytes * sizeof(valT), full + st);
      }
      if (diag && whole) bulk_g2s(s_diag(st), diag + r0, TR * sizeof(valT), full + st);
      if (STAGE_VEC) {
        const size_t voff = (size_t)r0 * R * 2;
        if (!FIRST) bulk_g2s(s_vec(st, 0), prev + voff, static_cast<uint32_t>(G::kVecBytes), full + st);
        if (!DBL) bulk_g2s(s_vec(st, 1), v0 + voff, static_cast<uint32_t>(G::kVecBytes), full + st);
      }
    }
  };

  const int64_t my_tiles = walk.count();
  int64_t run_head = tile_of(0);
  int64_t issued = 0;
  if (threadIdx.x < 32)
    for (; issued < my_tiles && issued < STAGES; ++issued) issue(issued);

  DotAcc<real> acc[CPT], acc2[CPT];
  bool ok = true;
  int64_t kk = 0;
  for (; kk < my_tiles; ++kk) {
    const int st = static_cast<int>(kk % STAGES);
    const uint32_t parity = static_cast<uint32_t>((kk / STAGES) & 1);
    ok = __syncthreads_and(mbar_wait_bounded(full + st, parity)) != 0;
    if (!ok) break;
    const int64_t tile = tile_of(kk);
    const int64_t r0 = tile * TR;
    const int64_t *hdr = s_hdr(st);
    const int64_t e0 = hdr[0];
    const bool bulk = (hdr[G::kSlices] - e0) <= G::kEl;
    const bool whole = r0 + TR <= n;
#pragma unroll 1
    for (int q = 0; q < RPT; ++q) {
      const int lr = lr0 + q * TRW;
      const int64_t i = r0 + lr;
      if (i < n) {
        const int64_t off = (i * R + part * CPT) * 2;
        real p[2 * CPT], z[2 * CPT];
        if (STAGE_VEC) {
          const int loff = (lr * R + part * CPT) * 2;
          if (!FIRST) memcpy(p, s_vec(st, 0) + loff, sizeof(p));
          if (!DBL) memcpy(z, s_vec(st, 1) + loff, sizeof(z));
        } else {
          if (!FIRST) ld_stream<real, CPT>(prev + off, p);
          if (!DBL) ld_stream<real, CPT>(v0 + off, z);
        }
        real d = real(0);
        if (diag) d = whole ? static_cast<real>(s_diag(st)[lr]) : static_cast<real>(__ldg(diag + i));
        d -= shift;
        const int64_t sb = hdr[lr >> 5];
        const int w = static_cast<int>((hdr[(lr >> 5) + 1] - sb) >> 5);
        real y[2 * CPT];
#pragma unroll
        for (int c = 0; c < 2 * CPT; ++c) y[c] = real(0);
        if (bulk) {
          const int32_t *cs = s_col(st) + (sb - e0) + (lr & 31);
          const valT *vs = s_val(st) + (sb - e0) + (lr & 31);
          if (w <= 12) {
            row_product_smem<real, valT, R, CPT, 12>(cs, vs, xp, w, y);
          } else {
#pragma unroll 1
            for (int s2 = 0; s2 < w; ++s2) {
              real xv[2 * CPT];
              const real h = static_cast<real>(vs[32 * s2]);
              ld_gather<real, CPT>(xp + (int64_t)cs[32 * s2] * (R * 2), xv);
#pragma unroll
              for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(h, xv[c], y[c]);
            }
          }
        } else {
          row_product_direct<real, valT, R, CPT>(col, val, x, sb + (i & 31), w, part, y);
        }
        real xi[2 * CPT];
        ld_gather<real, CPT>(x + off, xi);
        row_finish<real, CPT, FIRST, DBL>(y, xi, p, z, d, alpha, out + off, acc, acc2);
      }
    }
    if (SEG)
      segment_boundary<real, R, CPT, DBL>(acc, acc2, partial, slot_stride, bt, tile, TR,
                                          kk + 1 < my_tiles ? tile_of(kk + 1) : -1, run_head);
    __syncthreads();  // every thread is done with this stage
    if (threadIdx.x < 32 && issued < my_tiles) issue(issued++);
  }
  if (!ok) {
    if (threadIdx.x == 0) {
      atomicOr(flags, 4);
      for (int64_t q = kk; q < issued; ++q)
        mbar_wait_bounded(full + q % STAGES, static_cast<uint32_t>((q / STAGES) & 1));
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[c] = acc2[c] = DotAcc<real>();
  }
  if (!SEG) flush_partials<real, R, CPT, DBL>(acc, acc2, partial, blockIdx.x, slot_stride);
}

// ---------------------------------------------------------------------------
// Banded step (kind 3 shapes; needs the plan of kpm_band.cuh for T =
// kBlock / TPR).  A stage holds the tile's record, its local indices and
// values (kBandSlots slots per row at most), its diagonal (whole tiles), its
// streamed rows of v_{n-1} (and v0) and the ROWS x rows of its bands.  The
// producer (thread 0) keeps the records one tile ahead in a two-entry ring of
// its own, so that it knows the bands of a tile when it refills a stage.
// Tiles with nb < 0 stream only the vector rows and gather from global.
// ---------------------------------------------------------------------------
template <typename real, typename valT, int R, int CPT, int STAGES, int ROWS, int NV>
struct BandGeom {
  static constexpr int TPR = R / CPT;
  static constexpr int TR = kBlock / TPR;
  static constexpr int kEl = TR * kBandSlots;
  static constexpr size_t kRowBytes = (size_t)R * 2 * sizeof(real);
  static constexpr size_t kRecBytes = sizeof(BandRec);
  static constexpr size_t kIdxBytes = (kEl * 2 + 15) / 16 * 16;
  static constexpr size_t kValBytes = kEl * sizeof(valT);
  static constexpr size_t kDiagBytes = (TR * sizeof(valT) + 15) / 16 * 16;
  static constexpr size_t kVecBytes = (size_t)TR * kRowBytes;
  static constexpr size_t kXBytes = (size_t)ROWS * kRowBytes;
  static constexpr size_t kStageBytes = kRecBytes + kIdxBytes + kValBytes + kDiagBytes + NV * kVecBytes + kXBytes;
  static constexpr size_t kSmem = 256 + 2 * kRecBytes + STAGES * kStageBytes;   // barriers, record ring
  static constexpr bool kOk = TR % 32 == 0 && TR / 32 + 1 <= 9 && kSmem <= 220 * 1024 && STAGES >= 2 &&
                              STAGES <= 4 && ROWS <= 65535;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// FREE: no CTA barrier per tile; each warp releases a stage on its "empty"
// mbarrier (8 arrivals), and warp 0 refills a stage once its previous tile
// is released by every warp, before waiting on its own next stage.
template <typename real, typename valT, int R, int CPT, int STAGES, int MINB, int ROWS, bool FREE, bool FIRST,
          bool DBL, bool SEG>
__global__ void __launch_bounds__(kBlock, MINB) cheb_step_band_kernel(
    int64_t n, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ col,
    const valT *__restrict__ val, const valT *__restrict__ diag, const real *__restrict__ x, const real *prev,
    const real *__restrict__ v0, real *out, double *__restrict__ partial, real alpha, real shift,
    int *__restrict__ flags, int64_t slot_stride, BatchTables bt, const BandRec *__restrict__ recs,
    const uint16_t *__restrict__ lidx) {
  using G = BandGeom<real, valT, R, CPT, STAGES, ROWS, DBL ? 1 : 2>;
  constexpr int TPR = G::TPR, TR = G::TR;
  constexpr int RE = R * 2;   // reals per x row
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smem);          // [STAGES]
  uint64_t *recbar = full + 8;                                  // [2]
  uint64_t *empty = full + 10;                                  // [STAGES] (FREE)
  BandRec *rring = reinterpret_cast<BandRec *>(smem + 256);     // [2]
  unsigned char *ring = smem + 256 + 2 * G::kRecBytes;
  auto s_rec = [&](int st) { return reinterpret_cast<BandRec *>(ring + st * G::kStageBytes); };
  auto s_idx = [&](int st) { return reinterpret_cast<uint16_t *>(ring + st * G::kStageBytes + G::kRecBytes); };
  auto s_val = [&](int st) {
    return reinterpret_cast<valT *>(ring + st * G::kStageBytes + G::kRecBytes + G::kIdxBytes);
  };
  auto s_diag = [&](int st) {
    return reinterpret_cast<valT *>(ring + st * G::kStageBytes + G::kRecBytes + G::kIdxBytes + G::kValBytes);
  };
  auto s_vec = [&](int st, int q) {
    return reinterpret_cast<real *>(ring + st * G::kStageBytes + G::kRecBytes + G::kIdxBytes + G::kValBytes +
                                    G::kDiagBytes + q * G::kVecBytes);
  };
  auto s_x = [&](int st) {
    return reinterpret_cast<real *>(ring + st * G::kStageBytes + G::kRecBytes + G::kIdxBytes + G::kValBytes +
                                    G::kDiagBytes + (DBL ? 1 : 2) * G::kVecBytes);
  };
  const int64_t ntiles = (n + TR - 1) / TR;
  const int part = threadIdx.x % TPR;
  const int lr = threadIdx.x / TPR;
  const TileWalk<SEG ? kSegChunk : 1> walk(ntiles);   // this CTA's tiles, in order
  auto tile_of = [&](int64_t kk) { return walk.tile(kk); };
  const int64_t my_tiles = walk.count();

  if (threadIdx.x == 0) {
    for (int st = 0; st < STAGES; ++st) mbar_init(full + st, 1);
    if (FREE)
      for (int st = 0; st < STAGES; ++st) mbar_init(empty + st, kWarps);
    mbar_init(recbar, 1);
    mbar_init(recbar + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  bool ok = true;   // warp 0: its record waits
  // producer side (warp 0): lane 0 keeps the records one tile ahead; after a
  // record arrives every lane reads it and the lanes issue the tile's copies
  // in parallel (lane b < nb: band b; lanes 8..12: indices, values, diagonal,
  // vector rows)
  const int lane = threadIdx.x & 31;
  auto fetch_rec = [&](int64_t kk) {   // record of local tile kk into the record ring (lane 0)
    const int slot = static_cast<int>(kk & 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(recbar + slot, sizeof(BandRec));
    bulk_g2s(rring + slot, recs + tile_of(kk), sizeof(BandRec), recbar + slot);
  };
  auto issue = [&](int64_t kk) -> bool {
    const int slot = static_cast<int>(kk & 1);
    const bool got = mbar_wait_bounded(recbar + slot, static_cast<uint32_t>((kk >> 1) & 1));
    if (!__all_sync(0xffffffffu, got)) {
      ok = false;
      return false;
    }
    const int64_t tile = tile_of(kk);
    const int st = static_cast<int>(kk % STAGES);
    const int64_t r0 = tile * TR;
    const BandRec &rc = rring[slot];
    BandRec *dst = s_rec(st);
    if (lane < 8) reinterpret_cast<int4 *>(dst)[lane] = reinterpret_cast<const int4 *>(&rc)[lane];
    const int nb = rc.nb;
    const bool banded = nb > 0;
    const bool whole = r0 + TR <= n;
    const uint32_t cnt = static_cast<uint32_t>(rc.srel[TR / 32 < 9 ? TR / 32 : 8]);
    const int lo_b = lane < kBandMax ? rc.lo[lane] : 0;
    const int len_b = lane < kBandMax ? rc.len[lane] : 0;
    const int off_b = lane < kBandMax ? rc.off[lane] : 0;
    const int64_t e0 = rc.e0;
    __syncwarp();   // every lane has read the ring slot and the stage record is written
    if (lane == 0) {
      uint32_t tx = static_cast<uint32_t>(G::kVecBytes) * ((FIRST ? 0u : 1u) + (DBL ? 0u : 1u));
      if (banded) {
        uint32_t xrows = 0;
        for (int b = 0; b < nb; ++b) xrows += static_cast<uint32_t>(rc.len[b]);
        tx += cnt * (2u + static_cast<uint32_t>(sizeof(valT))) + xrows * static_cast<uint32_t>(G::kRowBytes);
        if (diag && whole) tx += TR * sizeof(valT);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(full + st, tx);
      if (kk + 1 < my_tiles) fetch_rec(kk + 1);   // the ring slot of kk - 1 is free
    }
    __syncwarp();
    if (banded) {
      if (lane < nb)
        bulk_g2s(s_x(st) + (size_t)off_b * RE, x + (size_t)lo_b * RE,
                 static_cast<uint32_t>(len_b) * static_cast<uint32_t>(G::kRowBytes), full + st);
      if (lane == 8 && cnt > 0) bulk_g2s(s_idx(st), lidx + tile * (int64_t)TR * kBandSlots, cnt * 2u, full + st);
      if (lane == 9 && cnt > 0)
        bulk_g2s(s_val(st), val + e0, cnt * static_cast<uint32_t>(sizeof(valT)), full + st);
      if (lane == 10 && diag && whole) bulk_g2s(s_diag(st), diag + r0, TR * sizeof(valT), full + st);
    }
    const size_t voff = (size_t)r0 * RE;
    if (!FIRST && lane == 11) bulk_g2s(s_vec(st, 0), prev + voff, static_cast<uint32_t>(G::kVecBytes), full + st);
    if (!DBL && lane == 12) bulk_g2s(s_vec(st, 1), v0 + voff, static_cast<uint32_t>(G::kVecBytes), full + st);
    return true;
  };

  int64_t issued = 0;
  if (threadIdx.x < 32 && my_tiles > 0) {
    if (lane == 0) fetch_rec(0);
    while (issued < my_tiles && issued < STAGES && issue(issued)) ++issued;
  }

  int64_t run_head = tile_of(0);
  DotAcc<real> acc[CPT], acc2[CPT];
  int64_t kk = 0;
  for (; kk < my_tiles; ++kk) {
    const int st = static_cast<int>(kk % STAGES);
    const uint32_t parity = static_cast<uint32_t>((kk / STAGES) & 1);
    if (FREE) {
      if (threadIdx.x < 32) {
        // refill the stages up to tile kk + STAGES - 1, each once every warp
        // has released its previous tile
        while (ok && issued < my_tiles && issued <= kk + STAGES - 1) {
          const int64_t prev_use = issued / STAGES - 1;
          const bool freed = mbar_wait_bounded(empty + issued % STAGES, static_cast<uint32_t>(prev_use & 1));
          if (!__all_sync(0xffffffffu, freed) || !issue(issued)) {
            ok = false;
            break;
          }
          ++issued;
        }
      }
      const bool got = ok && mbar_wait_bounded(full + st, parity);
      ok = __all_sync(0xffffffffu, got);
    } else {
      const bool mine = threadIdx.x >= 32 || ok;
      ok = __syncthreads_and(mine && mbar_wait_bounded(full + st, parity)) != 0;
    }
    if (!ok) break;
    const int64_t tile = tile_of(kk);
    const int64_t r0 = tile * TR;
    const int64_t i = r0 + lr;
    if (i < n) {
      const BandRec &rc = *s_rec(st);
      const bool banded = rc.nb > 0;
      const int64_t off = (i * R + part * CPT) * 2;
      const int q = lr >> 5;
      const int sb = rc.srel[q];
      const int w = (rc.srel[q + 1] - sb) >> 5;
      real p[2 * CPT], z[2 * CPT];
      if (!FIRST) memcpy(p, s_vec(st, 0) + (lr * R + part * CPT) * 2, sizeof(p));
      if (!DBL) memcpy(z, s_vec(st, 1) + (lr * R + part * CPT) * 2, sizeof(z));
      real d = real(0);
      if (diag) d = (banded && r0 + TR <= n) ? static_cast<real>(s_diag(st)[lr]) : static_cast<real>(__ldg(diag + i));
      d -= shift;
      real y[2 * CPT];
#pragma unroll
      for (int c = 0; c < 2 * CPT; ++c) y[c] = real(0);
      real xi[2 * CPT];
      if (banded) {
        const real *xs = s_x(st) + part * CPT * 2;
        const uint16_t *li = s_idx(st) + sb + (lr & 31);
        const valT *vs = s_val(st) + sb + (lr & 31);
        // rows of slices at most 12 wide (graphene within 3 A) take a 12-slot
        // body; 64-register budgets (4 CTAs) keep four slots in flight
        auto slots = [&](auto wmax) {
          constexpr int W = decltype(wmax)::value;
#pragma unroll(MINB >= 4 ? 4 : W)
          for (int s = 0; s < W; ++s) {
            if (s < w) {
              real xv[2 * CPT];
              const real h = static_cast<real>(vs[32 * s]);
              memcpy(xv, xs + (int)li[32 * s] * RE, sizeof(xv));
#pragma unroll
              for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(h, xv[c], y[c]);
            }
          }
        };
        if (w <= 12) slots(std::integral_constant<int, 12>{});
        else slots(std::integral_constant<int, kBandSlots>{});
        memcpy(xi, xs + (rc.own + lr) * RE, sizeof(xi));
      } else {
        row_product_direct<real, valT, R, CPT>(col, val, x, rc.e0 + sb + (lr & 31), w, part, y);
        ld_gather<real, CPT>(x + off, xi);
      }
      row_finish<real, CPT, FIRST, DBL>(y, xi, p, z, d, alpha, out + off, acc, acc2);
    }
    if (SEG)
      segment_boundary<real, R, CPT, DBL>(acc, acc2, partial, slot_stride, bt, tile, TR,
                                          kk + 1 < my_tiles ? tile_of(kk + 1) : -1, run_head);
    if (FREE) {
      __syncwarp();
      if (lane == 0) mbar_arrive(empty + st);   // this warp is done with the stage
    } else {
      __syncthreads();  // every thread is done with this stage
      if (threadIdx.x < 32 && issued < my_tiles && ok && issue(issued)) ++issued;
    }
  }
  if (FREE) ok = __syncthreads_and(ok) != 0;   // a warp that gave up reports for the CTA
  if (!ok) {
    if (threadIdx.x == 0) {
      atomicOr(flags, 4);
      for (int64_t q = kk; q < issued; ++q)
        mbar_wait_bounded(full + q % STAGES, static_cast<uint32_t>((q / STAGES) & 1));
      if (issued < my_tiles) mbar_wait_bounded(recbar + (issued & 1), static_cast<uint32_t>((issued >> 1) & 1));
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[c] = acc2[c] = DotAcc<real>();
  }
  if (!SEG) flush_partials<real, R, CPT, DBL>(acc, acc2, partial, blockIdx.x, slot_stride);
}

// mu_r[r, m] = (sum over CTAs in index order of partial[m, cta, r]) / n;
// flags[0] |= 1 if |mu| > bound (when bound > 0), |= 2 if not finite.
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
                                     int doubling, double bound, double *__restrict__ mu_r, int *__restrict__ flags) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)M * R) return;
  const int m = static_cast<int>(t / R), r = static_cast<int>(t % R);
  double mu = slot_sum(partial, grid, R, m, r) * inv_n;
  if (doubling && m >= 2) mu = 2.0 * mu - slot_sum(partial, grid, R, m & 1, r) * inv_n;
  mu_r[(int64_t)r * M + m] = mu;
  if (!isfinite(mu)) atomicOr(flags, 2);
  else if (bound > 0.0 && fabs(mu) > bound) atomicOr(flags, 1);
}

// ---------------------------------------------------------------------------
// Launch shapes.  A shape fixes the kernel family (direct loads or the
// bulk-copy ring), the complex numbers per thread CPT (so TPR = R / CPT
// threads share a row), the ring depth and the resident CTAs per SM that the
// register budget is sized for (the minimum blocks of __launch_bounds__).
// Entry 0 of every list is the default; the autotuner (tb_kpm_autotune)
// times the whole list on the caller's matrix.  Every shape computes the
// same moments up to the grouping of the partial sums, and each is bitwise
// reproducible.
// ---------------------------------------------------------------------------
struct StepShape {
  int kind;        // 0: direct loads, 1: bulk-copy ring, 2: second ring (offsets, diagonal staged),
                   // 3: banded step (x bands staged; needs the band plan)
  int opt;         // options: ring 1 = 12-slot body; banded 1 = no CTA barrier per tile
  int cpt;         // complex numbers per thread
  int stages;      // ring depth (rings only)
  int minb;        // resident CTAs per SM of the register budget
  int rpt;         // rows per thread per tile (second ring; 1 otherwise)
  int svec;        // the ring stages v_{n-1} (and v0) rows in shared memory
  int brows;       // banded step: x rows a stage holds for the tile's bands
};
constexpr StepShape D(int cpt, int minb) { return {0, 0, cpt, 0, minb, 1, 0, 0}; }
constexpr StepShape P(int cpt, int stages, int minb, int opt = 0) { return {1, opt, cpt, stages, minb, 1, 1, 0}; }
constexpr StepShape Q(int cpt, int stages, int minb, int rpt, int svec) {
  return {2, 0, cpt, stages, minb, rpt, svec, 0};
}
constexpr StepShape B(int cpt, int stages, int minb, int brows, int opt = 0) {
  return {3, opt, cpt, stages, minb, 1, 1, brows};
}

template <typename real, int R> struct Shapes;
// FP32 vectors.  Entry 0 is the hand-picked default of the library's first
// version; the other entries are the ones that won or came close in the
// autotuner on GB300 (10M-atom R = 8, 1M-atom R = 16, 100M-atom R = 1):
// the 2-stage ring, the 12-slot ring, the banded step (fastest at R = 1 and,
// without CTA barriers, at R = 8).  Slower candidates that were measured and
// dropped are listed in the design notes.
template <> struct Shapes<float, 1> {
  static constexpr StepShape at[] = {D(1, 4), D(1, 3), B(1, 2, 3, 1024), B(1, 2, 3, 1024, 1)};
};
template <> struct Shapes<float, 2> {
  static constexpr StepShape at[] = {D(2, 3), D(1, 4)};
};
template <> struct Shapes<float, 4> {
  static constexpr StepShape at[] = {D(4, 2), D(2, 3), P(2, 3, 2), B(2, 2, 3, 512, 1)};
};
template <> struct Shapes<float, 8> {
  static constexpr StepShape at[] = {P(2, 3, 4), P(2, 2, 4), P(2, 3, 4, 1), D(2, 3), B(2, 2, 3, 320, 1)};
};
template <> struct Shapes<float, 16> {
  static constexpr StepShape at[] = {P(2, 3, 4), P(2, 2, 4), D(2, 3), B(2, 2, 3, 192), B(2, 2, 3, 192, 1)};
};
template <> struct Shapes<float, 32> {
  static constexpr StepShape at[] = {D(2, 3), P(4, 3, 2), D(4, 2)};
};
// FP64 vectors (the FP64 pipe, not HBM, limits these on GB300).
template <> struct Shapes<double, 1> {
  static constexpr StepShape at[] = {D(1, 2), D(1, 3)};
};
template <> struct Shapes<double, 2> {
  static constexpr StepShape at[] = {D(2, 2)};
};
template <> struct Shapes<double, 4> {
  static constexpr StepShape at[] = {D(2, 2), P(2, 3, 1)};
};
template <> struct Shapes<double, 8> {
  static constexpr StepShape at[] = {P(2, 3, 1), P(2, 3, 2), D(2, 2), Q(2, 3, 2, 1, 0)};
};
template <> struct Shapes<double, 16> {
  static constexpr StepShape at[] = {P(2, 3, 1), D(2, 2), Q(2, 3, 2, 1, 0)};
};
template <> struct Shapes<double, 32> {
  static constexpr StepShape at[] = {D(2, 2)};
};

template <typename real, int R>
constexpr int shape_count() {
  return static_cast<int>(sizeof(Shapes<real, R>::at) / sizeof(StepShape));
}

// Everything that depends on one shape: occupancy-derived grid, shared
// memory opt-in and the launches.
// Device tables of the banded step (kind 3): one record per tile and the
// tile-local column indices (built by band_plan_kernel).
struct BandPlan {
  const BandRec *recs = nullptr;
  const uint16_t *lidx = nullptr;
};

template <typename real, typename valT, int R, int CPT, int KIND, int STAGES, int MINB, int RPT, int SVEC, int OPT,
          int BROWS>
struct ShapeKit {
  static constexpr int TPR = R / CPT;
  static constexpr int RPB = (kBlock / TPR) * (KIND == 2 ? RPT : 1);   // rows per tile
  static constexpr int S = STAGES >= 2 ? STAGES : 2;
  template <bool DBL>
  using GB = BulkGeom<real, valT, R, CPT, S, DBL ? 1 : 2>;
  template <bool DBL>
  using G2 = Ring2Geom<real, valT, R, CPT, S, RPT, SVEC != 0, DBL ? 1 : 2>;
  template <bool DBL>
  using GBand = BandGeom<real, valT, R, CPT, S, (BROWS > 0 ? BROWS : 32), (DBL ? 1 : 2)>;
  template <bool DBL>
  static constexpr size_t smem() {
    return KIND == 1 ? GB<DBL>::kSmem : (KIND == 2 ? G2<DBL>::kSmem : (KIND == 3 ? GBand<DBL>::kSmem : 0));
  }
  // the banded step's x rows must start on 16-byte boundaries
  static constexpr int kRowAlign = (R * 2 * (int)sizeof(real)) % 16 == 0 ? 1 : 16 / (R * 2 * (int)sizeof(real));
  static_assert(R % CPT == 0 && TPR <= 32, "bad shape");
  static_assert(KIND != 1 || (GB<true>::kOk && GB<false>::kOk), "ring shape does not fit");
  static_assert(KIND != 2 || (G2<true>::kOk && G2<false>::kOk), "second-ring shape does not fit");
  static_assert(KIND != 3 || (GBand<true>::kOk && GBand<false>::kOk), "banded shape does not fit");

  template <bool FIRST, bool DBL, bool SEG>
  static auto kernel() {
    if constexpr (KIND == 1)
      return cheb_step_bulk_kernel<real, valT, R, CPT, S, MINB, OPT, FIRST, DBL, SEG>;
    else if constexpr (KIND == 2)
      return cheb_step_ring2_kernel<real, valT, R, CPT, S, MINB, RPT, SVEC != 0, FIRST, DBL, SEG>;
    else if constexpr (KIND == 3)
      return cheb_step_band_kernel<real, valT, R, CPT, S, MINB, (BROWS > 0 ? BROWS : 32), (OPT & 1) != 0, FIRST, DBL,
                                   SEG>;
    else
      return cheb_step_kernel<real, valT, R, CPT, MINB, FIRST, DBL, SEG>;
  }
  template <bool FIRST, bool DBL, bool SEG>
  static void opt_in() {
    if (KIND != 0)
      cudaFuncSetAttribute(kernel<FIRST, DBL, SEG>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem<DBL>());
  }
  // opt every ring instantiation into its shared-memory size (before any
  // stream capture)
  static void prepare() {
    static bool done = false;
    if (done) return;
    opt_in<true, false, false>();
    opt_in<true, true, false>();
    opt_in<false, false, false>();
    opt_in<false, true, false>();
    opt_in<true, false, true>();
    opt_in<true, true, true>();
    opt_in<false, false, true>();
    opt_in<false, true, true>();
    done = true;
  }
  // resident CTAs per SM (doubling mode streams one vector less per stage, so
  // its ring kernels may fit more CTAs)
  static int per_sm(bool dbl) {
    static int cache[2] = {0, 0};
    int &c = cache[dbl ? 1 : 0];
    if (c == 0) {
      int b = 0;
      prepare();
      const cudaError_t e =
          dbl ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel<false, true, false>(), kBlock, smem<true>())
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel<false, false, false>(), kBlock,
                                                              smem<false>());
      c = (e != cudaSuccess || b <= 0) ? MINB : b;
    }
    return c;
  }
  static int grid(int64_t n, bool dbl) {
    const int64_t need = (n + RPB - 1) / RPB;
    const int64_t cap = (int64_t)per_sm(dbl) * sm_count();
    return static_cast<int>(need < cap ? need : cap);
  }
  // the band plan of this shape's tiles (kind 3 only)
  static tb_status plan(int64_t n, int64_t rows_avail, const int64_t *slice_ptr, const int32_t *col, BandRec *recs,
                        uint16_t *lidx, cudaStream_t st) {
    if constexpr (KIND == 3) {
      const int64_t tiles = (n + RPB - 1) / RPB;
      const int64_t cap = (int64_t)sm_count() * 4;
      band_plan_kernel<RPB><<<(unsigned)(tiles < cap ? tiles : cap), 256, 0, st>>>(n, slice_ptr, col, BROWS, kRowAlign,
                                                                                   rows_avail, recs, lidx);
      TB_CHECK_LAUNCH();
    }
    return TB_OK;
  }
  template <bool FIRST, bool DBL, bool SEG>
  static tb_status step(int grid, int64_t n, const int64_t *slice_ptr, const int32_t *col, const valT *val,
                        const valT *diag, const real *x, const real *prev, const real *v0, real *out,
                        double *partial, real alpha, real shift, int *flags, int64_t slot_stride,
                        const BatchTables &bt, cudaStream_t st, const BandPlan &bp = BandPlan()) {
    if constexpr (KIND == 0)
      cheb_step_kernel<real, valT, R, CPT, MINB, FIRST, DBL, SEG><<<grid, kBlock, 0, st>>>(
          n, slice_ptr, col, val, diag, x, prev, v0, out, partial, alpha, shift, slot_stride, bt);
    else if constexpr (KIND == 3)
      cheb_step_band_kernel<real, valT, R, CPT, S, MINB, (BROWS > 0 ? BROWS : 32), (OPT & 1) != 0, FIRST, DBL, SEG>
          <<<grid, kBlock, smem<DBL>(), st>>>(
          n, slice_ptr, col, val, diag, x, prev, v0, out, partial, alpha, shift, flags, slot_stride, bt, bp.recs,
          bp.lidx);
    else
      kernel<FIRST, DBL, SEG>()<<<grid, kBlock, smem<DBL>(), st>>>(n, slice_ptr, col, val, diag, x, prev, v0, out,
                                                                  partial, alpha, shift, flags, slot_stride, bt);
    TB_CHECK_LAUNCH();
    return TB_OK;
  }
};

template <typename real, typename valT, int R, int I>
using KitOf = ShapeKit<real, valT, R, Shapes<real, R>::at[I].cpt, Shapes<real, R>::at[I].kind,
                       Shapes<real, R>::at[I].stages, Shapes<real, R>::at[I].minb, Shapes<real, R>::at[I].rpt,
                       Shapes<real, R>::at[I].svec, Shapes<real, R>::at[I].opt, Shapes<real, R>::at[I].brows>;

// Call f(KitOf<..., I>{}) for the runtime shape index `id`.
template <typename real, typename valT, int R, int I = 0, typename F>
auto visit_shape(int id, F &&f) -> decltype(f(KitOf<real, valT, R, 0>{})) {
  if constexpr (I + 1 < shape_count<real, R>()) {
    if (id != I) return visit_shape<real, valT, R, I + 1>(id, std::forward<F>(f));
  }
  return f(KitOf<real, valT, R, I>{});
}

// The step interface used by the KPM and conductivity runners: every call
// names its shape (an index into Shapes<real, R>, validated by the caller).
template <typename real, typename valT, int R>
struct StepKit {
  static constexpr int kShapes = shape_count<real, R>();
  // complex numbers per thread of the default shape (the conductivity's
  // own per-row kernels use it)
  static constexpr int CPT = Shapes<real, R>::at[0].cpt;
  static constexpr int64_t kRowPad = 256;   // vector blocks hold whole tiles of every shape

  static int grid(int shape, int64_t n, bool dbl) {
    return visit_shape<real, valT, R>(shape, [&](auto k) { return decltype(k)::grid(n, dbl); });
  }
  static int rows_per_block(int shape) {
    return visit_shape<real, valT, R>(shape, [](auto k) { return decltype(k)::RPB; });
  }
  static bool pipelined(int shape) { return Shapes<real, R>::at[shape].kind != 0; }
  static bool banded(int shape) { return Shapes<real, R>::at[shape].kind == 3; }
  // band-plan storage of the banded shapes (records of the smallest tile,
  // kBandSlots local indices per row of the padded rows)
  static size_t plan_records(int64_t n) {
    int t = kBlock;
    for (int s = 0; s < kShapes; ++s)
      if (banded(s)) t = std::min(t, rows_per_block(s));
    return (size_t)((n + t - 1) / t);
  }
  static bool any_banded() {
    for (int s = 0; s < kShapes; ++s)
      if (banded(s)) return true;
    return false;
  }
  static tb_status plan(int shape, int64_t n, int64_t rows_avail, const int64_t *slice_ptr, const int32_t *col,
                        BandRec *recs, uint16_t *lidx, cudaStream_t st) {
    return visit_shape<real, valT, R>(shape, [&](auto k) {
      return decltype(k)::plan(n, rows_avail, slice_ptr, col, recs, lidx, st);
    });
  }
  // the second ring and the banded step bulk-copy the diagonal too
  static bool stages_diag(int shape) { return Shapes<real, R>::at[shape].kind >= 2; }
  // the largest grid and the smallest block over every shape and mode, so that
  // a workspace sized once fits whichever shape a later call takes
  static int max_grid(int64_t n) {
    int g = 1;
    for (int s = 0; s < kShapes; ++s) g = std::max(g, std::max(grid(s, n, false), grid(s, n, true)));
    return g;
  }
  static int min_rows_per_block() {
    int r = kBlock;
    for (int s = 0; s < kShapes; ++s) r = std::min(r, rows_per_block(s));
    return r;
  }
  static void prepare(int shape) {
    visit_shape<real, valT, R>(shape, [](auto k) {
      decltype(k)::prepare();
      return 0;
    });
  }
  template <bool FIRST, bool DBL, bool SEG>
  static tb_status step(int shape, int grid, int64_t n, const int64_t *slice_ptr, const int32_t *col,
                        const valT *val, const valT *diag, const real *x, const real *prev, const real *v0,
                        real *out, double *partial, real alpha, real shift, int *flags, int64_t slot_stride,
                        const BatchTables &bt, cudaStream_t st, const BandPlan &bp = BandPlan()) {
    return visit_shape<real, valT, R>(shape, [&](auto k) {
      return decltype(k)::template step<FIRST, DBL, SEG>(grid, n, slice_ptr, col, val, diag, x, prev, v0, out,
                                                         partial, alpha, shift, flags, slot_stride, bt, st, bp);
    });
  }
};

}  // namespace
}  // namespace gputb
