// Cell-list neighbour search: N(i) of Eq. 1 (arXiv 2509.06525 Sec. 3) =
// every atom j != i with a periodic image closer than r_cut, written
// straight into the SELL-32 column layout of the Hamiltonian.
//
// Passes (all on the device, O(N)):
//  1. cell_bin      fractional coordinates -> cell id, per-cell counts
//  2. scan          cell offsets (exclusive prefix sum)
//  3. cell_scatter  atoms and SoA positions in cell order
//  4. count         per-row neighbour count cnt_i and n_i (r < r_count)
//  5. slice widths  max cnt over each 32-row slice, overflow check, scan
//  6. fill          sorted neighbour indices of each row into col
// Pairs are screened in FP32 with a safety margin; only candidates whose
// |d|^2 lies within a relative 4e-6 of r_cut^2 (or r_count^2) take the
// explicitly rounded FP64 test, so membership is decided as the FP64
// definition states at a fraction of the FP64 work (GB300's FP64 rate is low).
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

__global__ void cell_bin_kernel(const double *__restrict__ pos, int64_t n, Box B, Grid G, int32_t *__restrict__ cell,
                                unsigned long long *__restrict__ count, int *__restrict__ flags) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  if (!isfinite(x) || !isfinite(y) || !isfinite(z)) {
    atomicOr(flags, 4);
    cell[i] = 0;
    atomicAdd(count, 1ull);
    return;
  }
  double3 pw;
  int3 c;
  wrap_and_bin(B, G, x, y, z, pw, c);
  const int64_t id = cell_index(G, c.x, c.y, c.z);
  cell[i] = static_cast<int32_t>(id);
  atomicAdd(count + id, 1ull);
}

// atoms of each cell in cell order, with their wrapped positions (SoA)
__global__ void cell_scatter_kernel(const double *__restrict__ pos, int64_t n, Box B, Grid G,
                                    const int32_t *__restrict__ cell, unsigned long long *__restrict__ cursor,
                                    int32_t *__restrict__ atom, double *__restrict__ px, double *__restrict__ py,
                                    double *__restrict__ pz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double3 pw;
  int3 c;
  wrap_and_bin(B, G, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], pw, c);
  const int64_t slot = (int64_t)atomicAdd(cursor + cell[i], 1ull);
  atom[slot] = static_cast<int32_t>(i);
  px[slot] = pw.x;
  py[slot] = pw.y;
  pz[slot] = pw.z;
}

// Search parameters: thresholds on r^2 with FP32 safety margins.  A
// candidate's FP64 displacement d is rounded to FP32 and its FP32 |d|^2 is
// within a relative 1e-6 of the exact value, so |d|^2 < lo means inside,
// >= hi outside; only candidates between lo and hi take the explicitly
// rounded FP64 test ((dx*dx + dy*dy) + dz*dz < r^2).
struct Radii {
  double rc2, rn2;            // exact thresholds (r_count^2 < 0 disables)
  float rc_lo, rc_hi, rn_lo, rn_hi;
};

// Visit every neighbour j of atom i: f(j, within_r_count).  Neighbour cells
// are visited with the lattice shift of their periodic image, so a pair
// costs one FP64 difference per component; directions with fewer than 3
// cells visit every cell with shifts -1, 0, +1 (only one image of j can be
// within r_cut because the periodic widths are at least 2 r_cut).
template <typename F>
__device__ __forceinline__ void for_each_neighbor(const Box &B, const Grid &G, const int64_t *__restrict__ start,
                                                  const int32_t *__restrict__ atom, const double *__restrict__ px,
                                                  const double *__restrict__ py, const double *__restrict__ pz,
                                                  int64_t i, const double3 &pwi, const int3 &ci, const Radii &rad,
                                                  F &&f) {
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
        const double s1 = shifts[0][q1], s2 = shifts[1][q2], s3 = shifts[2][q3];
        // q = pw_i - S: the displacement to the image of j is pw_j - q
        const double qx = pwi.x - (s1 * B.ax + s2 * B.bx + s3 * B.cx);
        const double qy = pwi.y - (s2 * B.by + s3 * B.cy);
        const double qz = pwi.z - s3 * B.cz;
        const int64_t c = cell_index(G, cells[0][q1], cells[1][q2], cells[2][q3]);
        const int64_t a0 = __ldg(start + c), a1 = __ldg(start + c + 1);
        for (int64_t s = a0; s < a1; ++s) {
          const double dx = __dsub_rn(__ldg(px + s), qx);
          const double dy = __dsub_rn(__ldg(py + s), qy);
          const double dz = __dsub_rn(__ldg(pz + s), qz);
          const float fx = static_cast<float>(dx), fy = static_cast<float>(dy), fz = static_cast<float>(dz);
          const float r2f = fx * fx + fy * fy + fz * fz;
          if (r2f >= rad.rc_hi) continue;
          const int32_t j = __ldg(atom + s);
          if (j == i) continue;
          double r2 = -1.0;
          if (r2f >= rad.rc_lo) {
            r2 = sq_norm(make_double3(dx, dy, dz));
            if (!(r2 < rad.rc2)) continue;
          }
          bool close = false;
          if (rad.rn2 > 0.0) {
            if (r2f < rad.rn_lo) close = true;
            else if (r2f < rad.rn_hi) {
              if (r2 < 0.0) r2 = sq_norm(make_double3(dx, dy, dz));
              close = r2 < rad.rn2;
            }
          }
          f(j, close);
        }
      }
}

__global__ void count_kernel(const double *__restrict__ pos, int64_t n, Box B, Grid G,
                             const int64_t *__restrict__ start, const int32_t *__restrict__ atom,
                             const double *__restrict__ px, const double *__restrict__ py,
                             const double *__restrict__ pz, Radii rad, int32_t *__restrict__ cnt,
                             int32_t *__restrict__ ncount) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double3 pwi;
  int3 ci;
  wrap_and_bin(B, G, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], pwi, ci);
  int c = 0, nc = 0;
  for_each_neighbor(B, G, start, atom, px, py, pz, i, pwi, ci, rad, [&](int32_t, bool close) {
    ++c;
    if (close) ++nc;
  });
  cnt[i] = c;
  if (ncount) ncount[i] = nc;
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

__global__ void fill_kernel(const double *__restrict__ pos, int64_t n, int64_t n_slices, Box B, Grid G,
                            const int64_t *__restrict__ start, const int32_t *__restrict__ atom,
                            const double *__restrict__ px, const double *__restrict__ py,
                            const double *__restrict__ pz, Radii rad, const int64_t *__restrict__ slice_ptr,
                            int32_t *__restrict__ col) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_slices * 32) return;
  const int64_t k = i >> 5;
  const int64_t base = slice_ptr[k] + (i & 31);
  const int w = static_cast<int>((slice_ptr[k + 1] - slice_ptr[k]) >> 5);
  if (i >= n) {  // phantom rows of the last slice
    for (int s = 0; s < w; ++s) col[base + 32 * s] = 0;
    return;
  }
  double3 pwi;
  int3 ci;
  wrap_and_bin(B, G, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], pwi, ci);
  int32_t list[kMaxWidth];
  int m = 0;
  for_each_neighbor(B, G, start, atom, px, py, pz, i, pwi, ci, rad, [&](int32_t j, bool) {
    if (m < w) {  // insertion sort, ascending j
      int p = m++;
      while (p > 0 && list[p - 1] > j) {
        list[p] = list[p - 1];
        --p;
      }
      list[p] = j;
    }
  });
  for (int s = 0; s < w; ++s) col[base + 32 * s] = s < m ? list[s] : static_cast<int32_t>(i);
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
  int32_t *cell, *atom;
  unsigned long long *count, *cursor;
  double *px, *py, *pz;
  int64_t *sizes, *total;
  int *flags;
  void *scan_ws;
};

size_t carve(Carver &cv, int64_t n, int64_t ncell, NeighborWs *w) {
  const int64_t n_slices = (n + 31) / 32;
  w->cell = cv.take<int32_t>(n);
  w->atom = cv.take<int32_t>(n);
  w->count = cv.take<unsigned long long>(ncell + 1);
  w->cursor = cv.take<unsigned long long>(ncell + 1);
  w->px = cv.take<double>(n);
  w->py = cv.take<double>(n);
  w->pz = cv.take<double>(n);
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

extern "C" size_t tb_neighbors_workspace_size(int64_t n, const double *box, const int32_t *pbc, double rcut) {
  Box B;
  if (n <= 0 || !(rcut > 0.0) || make_box(box, pbc, rcut, &B) != TB_OK) return 0;
  const Grid G = make_grid(B, rcut);
  Carver cv(nullptr, 0);
  NeighborWs w;
  return carve(cv, n, G.ncell, &w) + 256;
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
  carve(cv, n, G.ncell, &w);
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
  cell_bin_kernel<<<nb, 256, 0, st>>>(positions, n, B, G, w.cell, w.count, w.flags);
  TB_CHECK_LAUNCH();
  int64_t *start = reinterpret_cast<int64_t *>(w.count);
  s = exclusive_scan_i64(start, start, G.ncell + 1, w.total, w.scan_ws, st);
  if (s != TB_OK) return s;
  TB_CUDA(cudaMemcpyAsync(w.cursor, w.count, (G.ncell + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  cell_scatter_kernel<<<nb, 256, 0, st>>>(positions, n, B, G, w.cell, w.cursor, w.atom, w.px, w.py, w.pz);
  TB_CHECK_LAUNCH();
  count_kernel<<<nb, 256, 0, st>>>(positions, n, B, G, start, w.atom, w.px, w.py, w.pz, rad, cnt, ncount);
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
  if (hflags & 1) return fail(TB_ERR_ELL_OVERFLOW, "tb_build_neighbors: a row has more than %d neighbours", max_width);
  if (total > col_capacity || (total > 0 && !col))
    return fail(TB_ERR_ELL_OVERFLOW, "tb_build_neighbors: col needs %lld elements, capacity %lld", (long long)total,
                (long long)col_capacity);
  if (total > 0) {
    fill_kernel<<<(unsigned)((n_slices * 32 + 255) / 256), 256, 0, st>>>(
        positions, n, n_slices, B, G, start, w.atom, w.px, w.py, w.pz, rad, slice_ptr, col);
    TB_CHECK_LAUNCH();
  }
  return TB_OK;
}
