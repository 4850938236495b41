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
// Distances use the explicitly rounded FP64 minimum image of geometry.cuh,
// so membership is decided exactly as the FP64 definition states.
#include <cmath>

#include "geometry.cuh"

namespace gputb {

tb_status make_box(const double *b, const int32_t *pbc, double rcut, Box *out) {
  TB_REQUIRE(b && pbc, "box and pbc are required");
  for (int k = 0; k < 9; ++k) TB_REQUIRE(std::isfinite(b[k]), "box entries must be finite");
  if (b[1] != 0.0 || b[2] != 0.0 || b[5] != 0.0)
    return fail(TB_ERR_BOX, "box rows must have the form a1=(ax,0,0), a2=(bx,by,0), a3=(cx,cy,cz)");
  if (!(b[0] > 0.0 && b[4] > 0.0 && b[8] > 0.0)) return fail(TB_ERR_BOX, "box needs ax, by, cz > 0");
  Box B{b[0], b[3], b[4], b[6], b[7], b[8], pbc[0] != 0, pbc[1] != 0, pbc[2] != 0};
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

__device__ __forceinline__ int cell_coord(double s, int nc, int periodic) {
  if (!periodic || nc == 1) return 0;
  s = s - floor(s);
  int c = static_cast<int>(s * nc);
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__device__ __forceinline__ int3 cell_of(const Box &B, const Grid &G, double x, double y, double z) {
  const double s3 = z / B.cz;
  const double s2 = (y - s3 * B.cy) / B.by;
  const double s1 = (x - s3 * B.cx - s2 * B.bx) / B.ax;
  return make_int3(cell_coord(s1, G.nc[0], B.p1), cell_coord(s2, G.nc[1], B.p2), cell_coord(s3, G.nc[2], B.p3));
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
  const int3 c = cell_of(B, G, x, y, z);
  const int64_t id = cell_index(G, c.x, c.y, c.z);
  cell[i] = static_cast<int32_t>(id);
  atomicAdd(count + id, 1ull);
}

__global__ void cell_scatter_kernel(const double *__restrict__ pos, int64_t n, const int32_t *__restrict__ cell,
                                    unsigned long long *__restrict__ cursor, int32_t *__restrict__ atom,
                                    double *__restrict__ px, double *__restrict__ py, double *__restrict__ pz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t slot = (int64_t)atomicAdd(cursor + cell[i], 1ull);
  atom[slot] = static_cast<int32_t>(i);
  px[slot] = pos[3 * i];
  py[slot] = pos[3 * i + 1];
  pz[slot] = pos[3 * i + 2];
}

// Visit every candidate j of atom i (each candidate cell once), calling
// f(j, d, r2) for j != i with r2 < rcut2.
template <typename F>
__device__ __forceinline__ void for_each_neighbor(const Box &B, const Grid &G, const int64_t *__restrict__ start,
                                                  const int32_t *__restrict__ atom, const double *__restrict__ px,
                                                  const double *__restrict__ py, const double *__restrict__ pz,
                                                  int64_t i, double xi, double yi, double zi, int32_t my_cell,
                                                  double rcut2, F &&f) {
  const int c1 = (int)(my_cell % G.nc[0]);
  const int c2 = (int)((my_cell / G.nc[0]) % G.nc[1]);
  const int c3 = (int)(my_cell / ((int64_t)G.nc[0] * G.nc[1]));
  // search ranges: +-1 cell, or every cell when a direction has < 3 cells
  int lo[3], hi[3];
  const int cc[3] = {c1, c2, c3};
  for (int k = 0; k < 3; ++k) {
    if (G.nc[k] < 3) {
      lo[k] = 0;
      hi[k] = G.nc[k] - 1;
    } else {
      lo[k] = cc[k] - 1;
      hi[k] = cc[k] + 1;
    }
  }
  for (int d3 = lo[2]; d3 <= hi[2]; ++d3) {
    const int e3 = G.nc[2] < 3 ? d3 : (d3 + G.nc[2]) % G.nc[2];
    for (int d2 = lo[1]; d2 <= hi[1]; ++d2) {
      const int e2 = G.nc[1] < 3 ? d2 : (d2 + G.nc[1]) % G.nc[1];
      for (int d1 = lo[0]; d1 <= hi[0]; ++d1) {
        const int e1 = G.nc[0] < 3 ? d1 : (d1 + G.nc[0]) % G.nc[0];
        const int64_t c = cell_index(G, e1, e2, e3);
        const int64_t s0 = __ldg(start + c), s1 = __ldg(start + c + 1);
        for (int64_t s = s0; s < s1; ++s) {
          const int32_t j = __ldg(atom + s);
          if (j == i) continue;
          double3 d;
          d.x = __dsub_rn(__ldg(px + s), xi);
          d.y = __dsub_rn(__ldg(py + s), yi);
          d.z = __dsub_rn(__ldg(pz + s), zi);
          d = min_image(B, d);
          const double r2 = sq_norm(d);
          if (r2 < rcut2) f(j, r2);
        }
      }
    }
  }
}

__global__ void count_kernel(const double *__restrict__ pos, int64_t n, Box B, Grid G,
                             const int32_t *__restrict__ cell, const int64_t *__restrict__ start,
                             const int32_t *__restrict__ atom, const double *__restrict__ px,
                             const double *__restrict__ py, const double *__restrict__ pz, double rcut2,
                             double rcount2, int32_t *__restrict__ cnt, int32_t *__restrict__ ncount) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = 0, nc = 0;
  for_each_neighbor(B, G, start, atom, px, py, pz, i, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], cell[i], rcut2,
                    [&](int32_t, double r2) {
                      ++c;
                      if (r2 < rcount2) ++nc;
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
                            const int32_t *__restrict__ cell, const int64_t *__restrict__ start,
                            const int32_t *__restrict__ atom, const double *__restrict__ px,
                            const double *__restrict__ py, const double *__restrict__ pz, double rcut2,
                            const int64_t *__restrict__ slice_ptr, int32_t *__restrict__ col) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_slices * 32) return;
  const int64_t k = i >> 5;
  const int64_t base = slice_ptr[k] + (i & 31);
  const int w = static_cast<int>((slice_ptr[k + 1] - slice_ptr[k]) >> 5);
  if (i >= n) {  // phantom rows of the last slice
    for (int s = 0; s < w; ++s) col[base + 32 * s] = 0;
    return;
  }
  int32_t list[kMaxWidth];
  int m = 0;
  for_each_neighbor(B, G, start, atom, px, py, pz, i, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], cell[i], rcut2,
                    [&](int32_t j, double) {
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
  const double rc2 = rcut * rcut;
  const double rn2 = r_count > 0.0 ? r_count * r_count : -1.0;

  TB_CUDA(cudaMemsetAsync(w.count, 0, (G.ncell + 1) * sizeof(unsigned long long), st));
  TB_CUDA(cudaMemsetAsync(w.flags, 0, 4 * sizeof(int), st));
  cell_bin_kernel<<<nb, 256, 0, st>>>(positions, n, B, G, w.cell, w.count, w.flags);
  TB_CHECK_LAUNCH();
  int64_t *start = reinterpret_cast<int64_t *>(w.count);
  s = exclusive_scan_i64(start, start, G.ncell + 1, w.total, w.scan_ws, st);
  if (s != TB_OK) return s;
  TB_CUDA(cudaMemcpyAsync(w.cursor, w.count, (G.ncell + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  cell_scatter_kernel<<<nb, 256, 0, st>>>(positions, n, w.cell, w.cursor, w.atom, w.px, w.py, w.pz);
  TB_CHECK_LAUNCH();
  count_kernel<<<nb, 256, 0, st>>>(positions, n, B, G, w.cell, start, w.atom, w.px, w.py, w.pz, rc2, rn2, cnt,
                                   ncount);
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
        positions, n, n_slices, B, G, w.cell, start, w.atom, w.px, w.py, w.pz, rc2, slice_ptr, col);
    TB_CHECK_LAUNCH();
  }
  return TB_OK;
}
