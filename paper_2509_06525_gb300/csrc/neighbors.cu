// Cell-list neighbour search: N(i) of Eq. 1 (arXiv 2509.06525 Sec. 3) =
// every atom j != i with a periodic image closer than r_cut, written
// straight into the SELL-32 column layout of the Hamiltonian.
//
// Passes (all on the device, O(N)):
//  1. cell_bin      wrapped position and cell of every atom, per-cell counts
//  2. scan          cell offsets (exclusive prefix sum)
//  3. cell_scatter  positions in cell order: FP64, and split into two floats
//  4. search        one thread per row: neighbour count cnt_i, n_i
//                   (r < r_count) and the row's sorted list, once
//  5. slice widths  max cnt over each 32-row slice, overflow check, scan
//  6. compact       the sorted lists into the SELL-32 column array
// Pairs are screened in FP32: positions are stored as float pairs hi + lo
// (hi = fl32(x), lo = fl32(x - hi)) so that the difference of two nearby
// atoms is formed as (hi_j - hi_i) + (lo_j - lo_i) to a few FP32 ulps of
// |d| whatever the coordinates' magnitude.  Only candidates whose |d|^2
// lies within a relative 4e-6 of r_cut^2 (or r_count^2) take the explicitly
// rounded FP64 test, so membership is decided as the FP64 definition states
// with almost no FP64 work (GB300's FP64 rate is low).
#include <algorithm>
#include <cmath>

#include "geometry.cuh"

namespace gputb {

tb_status make_box(const double *b, const int32_t *pbc, double rcut, Box *out) {
  TB_REQUIRE(b && pbc, "box and pbc are required");
  for (int k = 0; k < 9; ++k) TB_REQUIRE(std::isfinite(b[k]), "box entries must be finite");
  if (b[1] != 0.0 || b[2] != 0.0 || b[5] != 0.0)
    return fail(TB_ERR_BOX, "box rows must have the form a1=(ax,0,0), a2=(bx,by,0), a3=(cx,cy,cz)");
  if (!(b[0] > 0.0 && b[4] > 0.0 && b[8] > 0.0)) return fail(TB_ERR_BOX, "box needs ax, by, cz > 0");
  Box B{b[0], b[3], b[4], b[6], b[7], b[8], pbc[0] != 0, pbc[1] != 0, pbc[2] != 0, 1.0 / b[0], 1.0 / b[4],
        1.0 / b[8]};
  const double vol = B.ax * B.by * B.cz;
  const double w1 = vol / std::sqrt((B.by * B.cz) * (B.by * B.cz) + (B.bx * B.cz) * (B.bx * B.cz) +
                                    (B.bx * B.cy - B.by * B.cx) * (B.bx * B.cy - B.by * B.cx));
  const double w2 = vol / (B.ax * std::sqrt(B.cy * B.cy + B.cz * B.cz));
  const double w3 = B.cz;
  const double w[3] = {w1, w2, w3};
  const int p[3] = {B.p1, B.p2, B.p3};
  for (int k = 0; k < 3; ++k)
    if (p[k] && w[k] < 2.0 * rcut)
      return fail(TB_ERR_BOX, "periodic width %.6g along a%d is below 2*rcut=%.6g", w[k], k + 1, 2.0 * rcut);
  *out = B;
  return TB_OK;
}

namespace {

constexpr int kMaxWidth = 64;   // hard cap on slots per row (local sort buffer)
// |wrapped coordinate| <= kCoordRange * rcut keeps the float-pair screen
// within its margin (the pair split leaves 2^-48 |x| of each coordinate)
constexpr double kCoordRange = 1048576.0;

struct Grid {
  int nc[3];       // cells per direction
  int64_t ncell;
};

// Fractional coordinates s (B^T s = p for the lower-triangular box rows),
// the periodic image of p inside the cell (pw = p - sum_k floor(s_k) a_k
// over periodic k) and its cell.  The same function serves the binning and
// the search, so every atom's wrapped position is computed identically.
__device__ __forceinline__ void wrap_and_bin(const Box &B, const Grid &G, double x, double y, double z, double3 &pw,
                                             int3 &cell) {
  // explicitly rounded operations: every kernel gets bit-identical results
  const double s3 = __ddiv_rn(z, B.cz);
  const double s2 = __ddiv_rn(__dsub_rn(y, __dmul_rn(s3, B.cy)), B.by);
  const double s1 = __ddiv_rn(__dsub_rn(__dsub_rn(x, __dmul_rn(s3, B.cx)), __dmul_rn(s2, B.bx)), B.ax);
  const double n1 = B.p1 ? floor(s1) : 0.0, n2 = B.p2 ? floor(s2) : 0.0, n3 = B.p3 ? floor(s3) : 0.0;
  pw.x = __dsub_rn(__dsub_rn(__dsub_rn(x, __dmul_rn(n1, B.ax)), __dmul_rn(n2, B.bx)), __dmul_rn(n3, B.cx));
  pw.y = __dsub_rn(__dsub_rn(y, __dmul_rn(n2, B.by)), __dmul_rn(n3, B.cy));
  pw.z = __dsub_rn(z, __dmul_rn(n3, B.cz));
  auto coord = [](double f, int nc, int periodic) {
    if (!periodic || nc == 1) return 0;
    int c = static_cast<int>(__dmul_rn(f, (double)nc));
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
  };
  cell = make_int3(coord(__dsub_rn(s1, n1), G.nc[0], B.p1), coord(__dsub_rn(s2, n2), G.nc[1], B.p2),
                   coord(__dsub_rn(s3, n3), G.nc[2], B.p3));
}

__device__ __forceinline__ int64_t cell_index(const Grid &G, int c1, int c2, int c3) {
  return ((int64_t)c3 * G.nc[1] + c2) * G.nc[0] + c1;
}

// wrapped positions (input order) and cells; flags |= 4 for a non-finite
// position, |= 8 for a coordinate beyond the float-pair screen's range
__global__ void cell_bin_kernel(const double *__restrict__ pos, int64_t n, Box B, Grid G, double max_abs,
                                int32_t *__restrict__ cell, double *__restrict__ pw_out,
                                unsigned long long *__restrict__ count, int *__restrict__ flags) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  double3 pw = make_double3(0.0, 0.0, 0.0);
  int64_t id = 0;
  if (!isfinite(x) || !isfinite(y) || !isfinite(z)) {
    atomicOr(flags, 4);
  } else {
    int3 c;
    wrap_and_bin(B, G, x, y, z, pw, c);
    id = cell_index(G, c.x, c.y, c.z);
    if (fabs(pw.x) > max_abs || fabs(pw.y) > max_abs || fabs(pw.z) > max_abs) atomicOr(flags, 8);
  }
  cell[i] = static_cast<int32_t>(id);
  pw_out[3 * i] = pw.x;
  pw_out[3 * i + 1] = pw.y;
  pw_out[3 * i + 2] = pw.z;
  atomicAdd(count + id, 1ull);
}

// positions in cell order: FP64 (for the exact test) and as float pairs
// (hi.w carries the atom index); slot_of[i] = the slot of atom i
__global__ void cell_scatter_kernel(int64_t n, const int32_t *__restrict__ cell, const double *__restrict__ pw,
                                    unsigned long long *__restrict__ cursor, int32_t *__restrict__ slot_of,
                                    float4 *__restrict__ hi, float4 *__restrict__ lo, double *__restrict__ px,
                                    double *__restrict__ py, double *__restrict__ pz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t slot = (int64_t)atomicAdd(cursor + cell[i], 1ull);
  slot_of[i] = static_cast<int32_t>(slot);
  const double x = pw[3 * i], y = pw[3 * i + 1], z = pw[3 * i + 2];
  px[slot] = x;
  py[slot] = y;
  pz[slot] = z;
  const float xh = __double2float_rn(x), yh = __double2float_rn(y), zh = __double2float_rn(z);
  hi[slot] = make_float4(xh, yh, zh, __int_as_float(static_cast<int32_t>(i)));
  lo[slot] = make_float4(__double2float_rn(__dsub_rn(x, (double)xh)), __double2float_rn(__dsub_rn(y, (double)yh)),
                         __double2float_rn(__dsub_rn(z, (double)zh)), 0.0f);
}

// Search parameters: thresholds on r^2 with FP32 safety margins.  The FP32
// |d|^2 of a candidate is within a relative 1e-6 of the exact value (float
// pair differences, coordinates below 2^20 r_cut), so |d|^2 < lo means
// inside, >= hi outside; only candidates between lo and hi take the
// explicitly rounded FP64 test ((dx*dx + dy*dy) + dz*dz < r^2).
struct Radii {
  double rc2, rn2;            // exact thresholds (r_count^2 < 0 disables)
  float rc_lo, rc_hi, rn_lo, rn_hi;
};

// Visit every neighbour j of atom i: f(j, within_r_count).  Neighbour cells
// are visited with the lattice shift of their periodic image (q = pw_i - S,
// the displacement to the image of j is pw_j - q); directions with fewer
// than 3 cells visit every cell with shifts -1, 0, +1 (only one image of j
// can be within r_cut because the periodic widths are at least 2 r_cut).
template <typename F>
__device__ __forceinline__ void for_each_neighbor(const Box &B, const Grid &G, const int64_t *__restrict__ start,
                                                  const float4 *__restrict__ hi, const float4 *__restrict__ lo,
                                                  const double *__restrict__ px, const double *__restrict__ py,
                                                  const double *__restrict__ pz, int64_t i, const double3 &pwi,
                                                  const float4 &hi_i, const float4 &lo_i, const int3 &ci,
                                                  const Radii &rad, F &&f) {
  int cells[3][6], shifts[3][6], cnt[3];
  const int cc[3] = {ci.x, ci.y, ci.z};
  const int per[3] = {B.p1, B.p2, B.p3};
  for (int k = 0; k < 3; ++k) {
    const int nc = G.nc[k];
    cnt[k] = 0;
    if (!per[k]) {
      for (int e = 0; e < nc; ++e) {
        cells[k][cnt[k]] = e;
        shifts[k][cnt[k]++] = 0;
      }
    } else if (nc >= 3) {
      for (int dlt = -1; dlt <= 1; ++dlt) {
        const int raw = cc[k] + dlt;
        cells[k][cnt[k]] = (raw + nc) % nc;
        shifts[k][cnt[k]++] = raw < 0 ? -1 : (raw >= nc ? 1 : 0);
      }
    } else {
      for (int e = 0; e < nc; ++e)
        for (int sh = -1; sh <= 1; ++sh) {
          cells[k][cnt[k]] = e;
          shifts[k][cnt[k]++] = sh;
        }
    }
  }
  for (int q3 = 0; q3 < cnt[2]; ++q3)
    for (int q2 = 0; q2 < cnt[1]; ++q2)
      for (int q1 = 0; q1 < cnt[0]; ++q1) {
        const int s1 = shifts[0][q1], s2 = shifts[1][q2], s3 = shifts[2][q3];
        double qx = pwi.x, qy = pwi.y, qz = pwi.z;
        float hx = hi_i.x, hy = hi_i.y, hz = hi_i.z, lx = lo_i.x, ly = lo_i.y, lz = lo_i.z;
        if (s1 | s2 | s3) {  // image cell: FP64 q, then its float pair
          qx = pwi.x - ((double)s1 * B.ax + (double)s2 * B.bx + (double)s3 * B.cx);
          qy = pwi.y - ((double)s2 * B.by + (double)s3 * B.cy);
          qz = pwi.z - (double)s3 * B.cz;
          hx = __double2float_rn(qx);
          hy = __double2float_rn(qy);
          hz = __double2float_rn(qz);
          lx = __double2float_rn(__dsub_rn(qx, (double)hx));
          ly = __double2float_rn(__dsub_rn(qy, (double)hy));
          lz = __double2float_rn(__dsub_rn(qz, (double)hz));
        }
        const int64_t c = cell_index(G, cells[0][q1], cells[1][q2], cells[2][q3]);
        const int64_t a0 = __ldg(start + c), a1 = __ldg(start + c + 1);
        for (int64_t s = a0; s < a1; ++s) {
          const float4 h = __ldg(hi + s), l = __ldg(lo + s);
          const float fx = __fadd_rn(__fsub_rn(h.x, hx), __fsub_rn(l.x, lx));
          const float fy = __fadd_rn(__fsub_rn(h.y, hy), __fsub_rn(l.y, ly));
          const float fz = __fadd_rn(__fsub_rn(h.z, hz), __fsub_rn(l.z, lz));
          const float r2f = fx * fx + fy * fy + fz * fz;
          if (r2f >= rad.rc_hi) continue;
          const int32_t j = __float_as_int(h.w);
          if (j == i) continue;
          double r2 = -1.0;
          auto exact = [&]() {
            const double dx = __dsub_rn(__ldg(px + s), qx);
            const double dy = __dsub_rn(__ldg(py + s), qy);
            const double dz = __dsub_rn(__ldg(pz + s), qz);
            return sq_norm(make_double3(dx, dy, dz));
          };
          if (r2f >= rad.rc_lo) {
            r2 = exact();
            if (!(r2 < rad.rc2)) continue;
          }
          bool close = false;
          if (rad.rn2 > 0.0) {
            if (r2f < rad.rn_lo) close = true;
            else if (r2f < rad.rn_hi) {
              if (r2 < 0.0) r2 = exact();
              close = r2 < rad.rn2;
            }
          }
          f(j, close);
        }
      }
}

// One thread per row: count, n_i and the sorted list (first cap entries)
// into the fixed-width buffer list[slice][cap][32].
__global__ void search_kernel(int64_t n, Box B, Grid G, const int64_t *__restrict__ start,
                              const int32_t *__restrict__ cell, const int32_t *__restrict__ slot_of,
                              const float4 *__restrict__ hi, const float4 *__restrict__ lo,
                              const double *__restrict__ px, const double *__restrict__ py,
                              const double *__restrict__ pz, Radii rad, int cap, int32_t *__restrict__ cnt,
                              int32_t *__restrict__ ncount, int32_t *__restrict__ list) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t slot = slot_of[i];
  const int32_t id = cell[i];
  const int3 ci = make_int3(id % G.nc[0], (id / G.nc[0]) % G.nc[1], id / (G.nc[0] * G.nc[1]));
  const double3 pwi = make_double3(px[slot], py[slot], pz[slot]);
  const float4 hi_i = hi[slot], lo_i = lo[slot];
  int32_t lst[kMaxWidth];
  int m = 0, c = 0, nclose = 0;
  for_each_neighbor(B, G, start, hi, lo, px, py, pz, i, pwi, hi_i, lo_i, ci, rad, [&](int32_t j, bool close) {
    ++c;
    if (close) ++nclose;
    if (m < cap) {  // insertion sort, ascending j
      int p = m++;
      while (p > 0 && lst[p - 1] > j) {
        lst[p] = lst[p - 1];
        --p;
      }
      lst[p] = j;
    }
  });
  cnt[i] = c;
  if (ncount) ncount[i] = nclose;
  int32_t *dst = list + (i >> 5) * 32 * (int64_t)cap + (i & 31);
  for (int s = 0; s < m; ++s) dst[32 * s] = lst[s];
}

// slice width = 32 * max(cnt) over the slice; flags |= 1 on overflow
__global__ void slice_width_kernel(const int32_t *__restrict__ cnt, int64_t n, int64_t n_slices, int max_width,
                                   int64_t *__restrict__ sizes, int *__restrict__ flags) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_slices) return;
  int w = 0;
  for (int l = 0; l < 32; ++l) {
    const int64_t i = k * 32 + l;
    if (i < n) w = max(w, cnt[i]);
  }
  if (w > max_width) {
    atomicOr(flags, 1);
    w = max_width;
  }
  sizes[k] = 32 * (int64_t)w;
}

// sorted lists -> SELL-32 columns (padding col = i, phantom rows col 0)
__global__ void compact_kernel(int64_t n, int64_t n_slices, const int64_t *__restrict__ slice_ptr,
                               const int32_t *__restrict__ cnt, const int32_t *__restrict__ list, int cap,
                               int32_t *__restrict__ col) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_slices * 32) return;
  const int64_t k = i >> 5;
  const int64_t base = slice_ptr[k] + (i & 31);
  const int w = static_cast<int>((slice_ptr[k + 1] - slice_ptr[k]) >> 5);
  if (i >= n) {
    for (int s = 0; s < w; ++s) col[base + 32 * s] = 0;
    return;
  }
  const int m = cnt[i];
  const int32_t *src = list + k * 32 * (int64_t)cap + (i & 31);
  for (int s = 0; s < w; ++s) col[base + 32 * s] = s < m ? __ldcs(src + 32 * s) : static_cast<int32_t>(i);
}

__global__ void read_total_kernel(const int64_t *slice_ptr, int64_t n_slices, int64_t *dst) {
  *dst = slice_ptr[n_slices];
}

Grid make_grid(const Box &B, double rcut) {
  const double vol = B.ax * B.by * B.cz;
  const double w1 = vol / std::sqrt((B.by * B.cz) * (B.by * B.cz) + (B.bx * B.cz) * (B.bx * B.cz) +
                                    (B.bx * B.cy - B.by * B.cx) * (B.bx * B.cy - B.by * B.cx));
  const double w2 = vol / (B.ax * std::sqrt(B.cy * B.cy + B.cz * B.cz));
  const double w3 = B.cz;
  const double w[3] = {w1, w2, w3};
  const int p[3] = {B.p1, B.p2, B.p3};
  Grid G;
  G.ncell = 1;
  for (int k = 0; k < 3; ++k) {
    int nc = 1;
    if (p[k]) {
      // cells strictly wider than rcut (relative margin far above rounding)
      const double c = std::floor(w[k] / (rcut * (1.0 + 1e-10)));
      nc = c < 1.0 ? 1 : (c > 1.0e6 ? 1000000 : static_cast<int>(c));
    }
    G.nc[k] = nc;
    G.ncell *= nc;
  }
  return G;
}

struct NeighborWs {
  int32_t *cell, *slot_of;
  unsigned long long *count, *cursor;
  double *pw;             // [N][3] wrapped positions, input order (until the scatter)
  int32_t *list;          // [ceil(N/32)][cap][32] sorted lists (shares pw's bytes)
  double *px, *py, *pz;   // wrapped positions, cell order
  float4 *hi, *lo;        // the same as float pairs
  int64_t *sizes, *total;
  int *flags;
  void *scan_ws;
};

size_t carve(Carver &cv, int64_t n, int64_t ncell, int cap, NeighborWs *w) {
  const int64_t n_slices = (n + 31) / 32;
  w->cell = cv.take<int32_t>(n);
  w->slot_of = cv.take<int32_t>(n);
  w->count = cv.take<unsigned long long>(ncell + 1);
  w->cursor = cv.take<unsigned long long>(ncell + 1);
  const size_t shared = std::max<size_t>(3 * sizeof(double) * (size_t)n, sizeof(int32_t) * (size_t)n_slices * 32 * cap);
  char *u = cv.take<char>(shared);
  w->pw = reinterpret_cast<double *>(u);
  w->list = reinterpret_cast<int32_t *>(u);
  w->px = cv.take<double>(n);
  w->py = cv.take<double>(n);
  w->pz = cv.take<double>(n);
  w->hi = cv.take<float4>(n);
  w->lo = cv.take<float4>(n);
  w->sizes = cv.take<int64_t>(n_slices + 1);
  w->total = cv.take<int64_t>(4);
  w->flags = cv.take<int>(4);
  const int64_t m = ncell + 1 > n_slices + 1 ? ncell + 1 : n_slices + 1;
  w->scan_ws = cv.take<char>(scan_workspace_bytes(m));
  return cv.used;
}

}  // namespace
}  // namespace gputb

using namespace gputb;

extern "C" size_t tb_neighbors_workspace_size(int64_t n, const double *box, const int32_t *pbc, double rcut,
                                               int32_t max_width) {
  Box B;
  if (n <= 0 || !(rcut > 0.0) || max_width < 1 || max_width > kMaxWidth || make_box(box, pbc, rcut, &B) != TB_OK)
    return 0;
  const Grid G = make_grid(B, rcut);
  Carver cv(nullptr, 0);
  NeighborWs w;
  return carve(cv, n, G.ncell, max_width, &w) + 256;
}

extern "C" tb_status tb_build_neighbors(const double *positions, int64_t n, const double *box, const int32_t *pbc,
                                        double rcut, double r_count, int32_t max_width, int64_t *slice_ptr,
                                        int32_t *col, int64_t col_capacity, int32_t *cnt, int32_t *ncount,
                                        int64_t *total_out, void *workspace, size_t workspace_bytes,
                                        void *stream) {
  TB_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "tb_build_neighbors: n=%lld out of range", (long long)n);
  TB_REQUIRE(positions && slice_ptr && cnt && workspace && total_out, "tb_build_neighbors: null pointer argument");
  TB_REQUIRE(rcut > 0.0 && std::isfinite(rcut), "tb_build_neighbors: rcut must be positive");
  TB_REQUIRE(max_width >= 1 && max_width <= kMaxWidth, "tb_build_neighbors: max_width must be in [1, %d]",
             kMaxWidth);
  TB_REQUIRE((reinterpret_cast<uintptr_t>(workspace) & 255) == 0, "tb_build_neighbors: workspace alignment");
  Box B;
  tb_status s = make_box(box, pbc, rcut, &B);
  if (s != TB_OK) return s;
  const Grid G = make_grid(B, rcut);
  TB_REQUIRE(G.ncell < (int64_t(1) << 31), "tb_build_neighbors: too many cells");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carver cv(workspace, workspace_bytes);
  NeighborWs w;
  carve(cv, n, G.ncell, max_width, &w);
  if (!cv.ok()) return fail(TB_ERR_WORKSPACE, "tb_build_neighbors: workspace too small");
  const int64_t n_slices = (n + 31) / 32;
  const unsigned nb = (unsigned)((n + 255) / 256);
  Radii rad;
  rad.rc2 = rcut * rcut;
  rad.rn2 = r_count > 0.0 ? r_count * r_count : -1.0;
  rad.rc_lo = static_cast<float>(rad.rc2 * (1.0 - 4e-6));
  rad.rc_hi = static_cast<float>(rad.rc2 * (1.0 + 4e-6));
  rad.rn_lo = rad.rn2 > 0.0 ? static_cast<float>(rad.rn2 * (1.0 - 4e-6)) : -1.0f;
  rad.rn_hi = rad.rn2 > 0.0 ? static_cast<float>(rad.rn2 * (1.0 + 4e-6)) : -1.0f;

  TB_CUDA(cudaMemsetAsync(w.count, 0, (G.ncell + 1) * sizeof(unsigned long long), st));
  TB_CUDA(cudaMemsetAsync(w.flags, 0, 4 * sizeof(int), st));
  cell_bin_kernel<<<nb, 256, 0, st>>>(positions, n, B, G, kCoordRange * rcut, w.cell, w.pw, w.count, w.flags);
  TB_CHECK_LAUNCH();
  int64_t *start = reinterpret_cast<int64_t *>(w.count);
  s = exclusive_scan_i64(start, start, G.ncell + 1, w.total, w.scan_ws, st);
  if (s != TB_OK) return s;
  TB_CUDA(cudaMemcpyAsync(w.cursor, w.count, (G.ncell + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  cell_scatter_kernel<<<nb, 256, 0, st>>>(n, w.cell, w.pw, w.cursor, w.slot_of, w.hi, w.lo, w.px, w.py, w.pz);
  TB_CHECK_LAUNCH();
  search_kernel<<<nb, 256, 0, st>>>(n, B, G, start, w.cell, w.slot_of, w.hi, w.lo, w.px, w.py, w.pz, rad,
                                    max_width, cnt, ncount, w.list);
  TB_CHECK_LAUNCH();
  TB_CUDA(cudaMemsetAsync(w.sizes, 0, (n_slices + 1) * sizeof(int64_t), st));
  slice_width_kernel<<<(unsigned)((n_slices + 255) / 256), 256, 0, st>>>(cnt, n, n_slices, max_width, w.sizes,
                                                                          w.flags);
  TB_CHECK_LAUNCH();
  s = exclusive_scan_i64(w.sizes, slice_ptr, n_slices + 1, w.total + 1, w.scan_ws, st);
  if (s != TB_OK) return s;
  int64_t host[2] = {0, 0};
  int hflags = 0;
  TB_CUDA(cudaMemcpyAsync(host, w.total, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  TB_CUDA(cudaMemcpyAsync(&hflags, w.flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  TB_CUDA(cudaStreamSynchronize(st));
  const int64_t total = host[1];
  *total_out = total;
  if (hflags & 4) return fail(TB_ERR_NOT_FINITE, "tb_build_neighbors: non-finite position");
  if (hflags & 8)
    return fail(TB_ERR_INVALID_ARG, "tb_build_neighbors: a wrapped coordinate exceeds %g * rcut", kCoordRange);
  if (hflags & 1) return fail(TB_ERR_ELL_OVERFLOW, "tb_build_neighbors: a row has more than %d neighbours", max_width);
  if (total > col_capacity || (total > 0 && !col))
    return fail(TB_ERR_ELL_OVERFLOW, "tb_build_neighbors: col needs %lld elements, capacity %lld", (long long)total,
                (long long)col_capacity);
  if (total > 0) {
    compact_kernel<<<(unsigned)((n_slices * 32 + 255) / 256), 256, 0, st>>>(n, n_slices, slice_ptr, cnt, w.list,
                                                                            max_width, col);
    TB_CHECK_LAUNCH();
  }
  return TB_OK;
}
