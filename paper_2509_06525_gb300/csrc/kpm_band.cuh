// Banded Chebyshev step: a per-matrix plan and the step kernel that uses it.
//
// The plan splits the rows into tiles of T rows (T = the step's rows per
// tile).  For each tile it records the few contiguous ranges ("bands") of x
// rows that the tile's columns -- and the tile's own rows -- fall in, and
// replaces each column index by a 16-bit index into the concatenation of the
// bands.  In cell-ordered structures a tile needs three bands: its own cell
// row and the two neighbouring cell rows.  The step kernel then bulk-copies
// the bands together with the tile's local indices, values and streamed
// vector rows into a shared-memory ring, so that warps take every operand of
// a row from shared memory and never wait on a global gather.  A tile whose
// columns need more than kBandMax bands, more rows than the stage holds, or
// has a slice wider than kBandSlots takes the global-gather path instead (its
// record has nb = -1).  Internal linkage in each translation unit that includes it.
#pragma once

#include <climits>

#include "kpm_common.cuh"

namespace gputb {
namespace {
using namespace kpmdev;

constexpr int kBandMax = 6;   // bands per tile
constexpr int kBandSlots = 16;   // widest slice a banded tile may have (SELL slots)

struct __align__(16) BandRec {
  int64_t e0;                // first SELL element of the tile
  int32_t nb;                // bands; -1: the tile takes the global-gather path
  int32_t own;               // local row index of the tile's first row
  int32_t lo[kBandMax];      // first x row of each band
  int32_t len[kBandMax];     // rows of each band
  int32_t off[kBandMax];     // local index of each band's first row
  int32_t srel[10];          // the tile's slice offsets minus e0 (T / 32 + 1 <= 9 entries)
};
static_assert(sizeof(BandRec) == 128, "BandRec layout");

// One CTA of 256 threads per tile (grid-stride over tiles).  The tile's
// columns and its own rows are reduced to 8-row groups (col >> 3) in a
// shared-memory hash set; the distinct groups (at most kMaxGroups, else the
// tile takes the gather path) are sorted, and runs of adjacent groups become
// the bands, 8-row aligned.  row_align (1 or 2) divides 8, so every band copy
// starts on a 16-byte boundary; rows_avail: rows of the vector blocks (bands
// never pass it).
constexpr int kGroupShift = 3;
constexpr int kGroupHash = 2048;
constexpr int kMaxGroups = 512;
constexpr int kHashProbes = 64;

template <int T>
__global__ void __launch_bounds__(256) band_plan_kernel(int64_t n, const int64_t *__restrict__ slice_ptr,
                                                        const int32_t *__restrict__ col, int max_rows, int row_align,
                                                        int64_t rows_avail, BandRec *__restrict__ rec,
                                                        uint16_t *__restrict__ lidx) {
  __shared__ int32_t hset[kGroupHash];
  __shared__ int32_t key[kMaxGroups];
  __shared__ int32_t s_start[kBandMax + 2];
  __shared__ int s_count, s_nd, s_over;
  __shared__ BandRec s_rec;
  const int64_t ntiles = (n + T - 1) / T;
  const int64_t n_slices = (n + 31) >> 5;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = t * T;
    const int64_t k0 = r0 >> 5;
    const int64_t k1 = min(k0 + T / 32, n_slices);
    const int64_t e0 = slice_ptr[k0];
    const int64_t cnt = slice_ptr[k1] - e0;
    const int rows = static_cast<int>(min((int64_t)T, n - r0));
    if (threadIdx.x == 0) {
      s_rec.e0 = e0;
      s_rec.nb = -1;
      s_rec.own = 0;
      for (int q = 0; q < 10; ++q)
        s_rec.srel[q] = static_cast<int32_t>(q <= k1 - k0 ? slice_ptr[k0 + q] - e0 : cnt);
      s_count = 0;
      s_nd = 0;
      s_over = 0;
    }
    for (int k = threadIdx.x; k < kGroupHash; k += blockDim.x) hset[k] = -1;
    __syncthreads();
    bool banded = true;
    for (int q = 0; q < T / 32; ++q) banded = banded && s_rec.srel[q + 1] - s_rec.srel[q] <= 32 * kBandSlots;
    if (banded) {
      // the 8-row groups of the tile's columns (phantom lanes of the last
      // slice left out) and of its own rows, into the hash set
      for (int64_t k = threadIdx.x; k < cnt + rows; k += blockDim.x) {
        int32_t gk = -1;
        if (k < cnt) {
          int q = 0;
          while (q + 1 <= T / 32 && s_rec.srel[q + 1] <= k) ++q;
          const int64_t row = (k0 + q) * 32 + (k - s_rec.srel[q]) % 32;
          if (row < n) gk = col[e0 + k] >> kGroupShift;
        } else {
          gk = static_cast<int32_t>((r0 + (k - cnt)) >> kGroupShift);
        }
        if (gk < 0) continue;
        uint32_t h = (static_cast<uint32_t>(gk) * 2654435761u) >> 21;   // 11 bits: kGroupHash slots
        int probe = 0;
        for (; probe < kHashProbes; ++probe) {
          const int32_t cur = hset[h];
          if (cur == gk) break;
          if (cur == -1) {
            const int32_t old = atomicCAS(&hset[h], -1, gk);
            if (old == -1 || old == gk) break;
          }
          h = (h + 1) & (kGroupHash - 1);
        }
        if (probe == kHashProbes) s_over = 1;
      }
      __syncthreads();
      for (int k = threadIdx.x; k < kGroupHash; k += blockDim.x) {
        const int32_t v = hset[k];
        if (v >= 0) {
          const int slot = atomicAdd(&s_nd, 1);
          if (slot < kMaxGroups) key[slot] = v;
        }
      }
      __syncthreads();
      const int nd = s_nd;
      banded = s_over == 0 && nd <= kMaxGroups;
      if (banded) {
        int P = 1;
        while (P < nd) P <<= 1;
        for (int k = nd + threadIdx.x; k < P; k += blockDim.x) key[k] = INT_MAX;
        __syncthreads();
        // bitonic sort of the distinct groups, ascending
        for (int size = 2; size <= P; size <<= 1) {
          for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int k = threadIdx.x; k < P / 2; k += blockDim.x) {
              const int lo = 2 * k - (k & (stride - 1));
              const int hi = lo + stride;
              const bool up = (lo & size) == 0;
              const int32_t a = key[lo], b = key[hi];
              if ((a > b) == up) {
                key[lo] = b;
                key[hi] = a;
              }
            }
            __syncthreads();
          }
        }
        // band starts: the first group and every group not adjacent to its
        // predecessor
        for (int k = threadIdx.x; k < nd; k += blockDim.x) {
          if (k == 0 || key[k] > key[k - 1] + 1) {
            const int slot = atomicAdd(&s_count, 1);
            if (slot <= kBandMax) s_start[slot] = k;
          }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          int nb = s_count;
          if (nb > kBandMax) {
            nb = -1;
          } else {
            for (int a = 1; a < nb; ++a)   // insertion sort of the starts
              for (int b = a; b > 0 && s_start[b - 1] > s_start[b]; --b) {
                const int tmp = s_start[b];
                s_start[b] = s_start[b - 1];
                s_start[b - 1] = tmp;
              }
            s_start[nb] = nd;
            int m = 0, total = 0;
            int64_t prev_hi = -1;
            for (int b = 0; b < nb; ++b) {
              int64_t lo = (int64_t)key[s_start[b]] << kGroupShift;
              int64_t hi = ((int64_t)key[s_start[b + 1] - 1] + 1) << kGroupShift;
              lo = lo / row_align * row_align;
              hi = min((hi + row_align - 1) / row_align * row_align, rows_avail);
              if (m > 0 && lo <= prev_hi) {   // bands that touch merge
                const int64_t nhi = max(prev_hi, hi);
                total += static_cast<int>(nhi - prev_hi);
                s_rec.len[m - 1] = static_cast<int32_t>(nhi - s_rec.lo[m - 1]);
                prev_hi = nhi;
                continue;
              }
              s_rec.lo[m] = static_cast<int32_t>(lo);
              s_rec.len[m] = static_cast<int32_t>(hi - lo);
              s_rec.off[m] = total;
              total += static_cast<int>(hi - lo);
              prev_hi = hi;
              ++m;
            }
            nb = total <= max_rows ? m : -1;
            if (nb > 0) {
              for (int b = 0; b < nb; ++b)
                if (r0 >= s_rec.lo[b] && r0 < s_rec.lo[b] + s_rec.len[b])
                  s_rec.own = s_rec.off[b] + static_cast<int32_t>(r0 - s_rec.lo[b]);
            }
          }
          for (int b = (nb > 0 ? nb : 0); b < kBandMax; ++b) s_rec.lo[b] = s_rec.len[b] = s_rec.off[b] = 0;
          s_rec.nb = nb;
        }
      }
      __syncthreads();
      banded = s_rec.nb > 0;
    }
    if (banded) {
      // local index of every element (phantom lanes get 0; never read)
      uint16_t *out = lidx + t * (int64_t)T * kBandSlots;
      for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        const int32_t c = col[e0 + k];
        int32_t li = 0;
        for (int b = 0; b < s_rec.nb; ++b)
          if (c >= s_rec.lo[b] && c < s_rec.lo[b] + s_rec.len[b]) li = s_rec.off[b] + (c - s_rec.lo[b]);
        out[k] = static_cast<uint16_t>(li);
      }
    }
    if (threadIdx.x < 8) {
      const int4 *src = reinterpret_cast<const int4 *>(&s_rec);
      reinterpret_cast<int4 *>(rec + t)[threadIdx.x] = src[threadIdx.x];
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace gputb
