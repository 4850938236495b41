// Learned Hamiltonian: radial Chebyshev descriptors (Eq. 2), per-edge SiLU
// MLP 32 -> 64 -> 64 -> 2 on BF16 tensor cores (forward and backward), the
// loss of the form of Eq. 3 on Hamiltonian elements, AdamW (Sec. 2.1), and
// the assembly of the learned H into SELL-32 (arXiv 2509.06525 Sec. 3).
//
//   f_k(r)  = (T_k(2 (r/r_cut - 1)^2 - 1) + 1) / 2 * f_c(r),  k = 0..7
//   C_n(r)  = sum_k c^{Z_i Z_j}_{nk} f_k(r);   v_i = sum_j C_n(r_ij)
//   x_ij    = [C(r_ij), v_i, v_j, C(r_ij) * (v_i + v_j)]      (32 features)
//   y       = W3 silu(W2 silu(W1 xn + b1) + b2) + b3,  xn = (x - mean) * inv_std
//   H_ij    = (y0(i->j) + y0(j->i)) / 2,   eps_i = eps0[Z_i] + sum_j y1(i->j)
//
// Tensor-core mapping (mma.sync.m16n8k16, BF16 in, FP32 accumulate): a CTA of
// 4 warps owns a tile of 128 edges; each warp runs its 32 edges as two
// 16-row blocks.  The FP32 accumulators of one layer are re-packed in
// registers as the BF16 A operand of the next (the C fragment of two
// adjacent 8-column tiles is exactly the A fragment of one 16-column
// k-tile), so activations never leave registers in the forward pass.
// Weights are staged once per CTA in shared memory with padded rows
// (conflict-free 32-bit fragment loads).  The backward pass recomputes the
// forward, forms dz2, dz1 in registers, writes transposed BF16 tiles to
// shared memory and accumulates the weight gradients dW1, dW2 as MMAs with
// the 128 edges as the reduction dimension; per-CTA partial gradients are
// summed in CTA order by a second kernel (deterministic).
#include <cmath>
#include <cstddef>
#include <cstring>

#include <cuda_bf16.h>

#include "descriptor.cuh"
#include "geometry.cuh"
#include "tcgen05.cuh"

namespace gputb {
namespace {

constexpr int NF = 32, NH = 64;
// FP32 parameter vector layout
constexpr int OFF_W1 = 0, OFF_B1 = 2048, OFF_W2 = 2112, OFF_B2 = 6208, OFF_W3 = 6272, OFF_B3 = 6400;
constexpr int NPARAM = 6402;
// BF16 weight copy layout
constexpr int WB_W1 = 0, WB_W2 = 2048, WB_W3 = 6144, NWB = 6272;

constexpr int TILE = 128;           // edges per CTA tile
constexpr int kThreads = 128;       // 4 warps
constexpr int SX = 40;              // bf16 row stride of the x tile (32 + 8 pad)
constexpr int SW1 = 40, SW2 = 72, SW3 = 72;
constexpr int ST = TILE + 8;        // bf16 row stride of transposed tiles

using bf16 = __nv_bfloat16;

__device__ __forceinline__ uint32_t ld32(const bf16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ uint32_t smem_u32_generic(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  uint32_t u;
  memcpy(&u, &v, 4);
  return u;
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// logistic function as 1/2 + tanh(z/2)/2 with the single-instruction
// hardware tanh (relative error about 2^-11, far below the BF16 rounding of
// the activations it feeds); forward, backward and the learned-H kernels
// all use it, so training and inference see the same network
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sigm(float z) { return fmaf(0.5f, tanh_fast(0.5f * z), 0.5f); }
__device__ __forceinline__ float silu(float z) { return z * sigm(z); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = sigm(z);
  return s * (1.0f + z * (1.0f - s));
}

struct Weights {
  alignas(16) bf16 w1[NH * SW1];
  alignas(16) bf16 w2[NH * SW2];
  alignas(16) bf16 w3[8 * SW3];
  alignas(16) float b1[NH];
  alignas(16) float b2[NH];
  alignas(16) float b3[2];
};

// stage weights (BF16 copy) and biases (FP32 master) into shared memory
__device__ void stage_weights(Weights &S, const bf16 *__restrict__ wb, const float *__restrict__ p) {
  for (int k = threadIdx.x; k < NH * NF; k += blockDim.x) S.w1[(k / NF) * SW1 + k % NF] = wb[WB_W1 + k];
  for (int k = threadIdx.x; k < NH * NH; k += blockDim.x) S.w2[(k / NH) * SW2 + k % NH] = wb[WB_W2 + k];
  for (int k = threadIdx.x; k < 8 * NH; k += blockDim.x)
    S.w3[(k / NH) * SW3 + k % NH] = k < 2 * NH ? wb[WB_W3 + k] : __float2bfloat16(0.0f);
  for (int k = threadIdx.x; k < NH; k += blockDim.x) {
    S.b1[k] = p[OFF_B1 + k];
    S.b2[k] = p[OFF_B2 + k];
  }
  if (threadIdx.x < 2) S.b3[threadIdx.x] = p[OFF_B3 + threadIdx.x];
}

// Forward of one 16-row block starting at row rb of the x tile xs.
// Outputs: z1, z2 (FP32 pre-activations, C layout) and y (layer-3 C tile).
__device__ __forceinline__ void forward_block(const Weights &S, const bf16 *xs, int rb, float (&z1)[8][4],
                                              float (&z2)[8][4], float (&y)[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t xa[2][4];
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    xa[kk][0] = ld32(xs + (rb + g) * SX + 16 * kk + 2 * t);
    xa[kk][1] = ld32(xs + (rb + g + 8) * SX + 16 * kk + 2 * t);
    xa[kk][2] = ld32(xs + (rb + g) * SX + 16 * kk + 2 * t + 8);
    xa[kk][3] = ld32(xs + (rb + g + 8) * SX + 16 * kk + 2 * t + 8);
  }
#pragma unroll
  for (int nn = 0; nn < 8; ++nn) {
    const float bl = S.b1[8 * nn + 2 * t], bh = S.b1[8 * nn + 2 * t + 1];
    float c[4] = {bl, bh, bl, bh};
#pragma unroll
    for (int kk = 0; kk < 2; ++kk)
      mma_bf16(c, xa[kk], ld32(S.w1 + (8 * nn + g) * SW1 + 16 * kk + 2 * t),
               ld32(S.w1 + (8 * nn + g) * SW1 + 16 * kk + 2 * t + 8));
#pragma unroll
    for (int q = 0; q < 4; ++q) z1[nn][q] = c[q];
  }
  uint32_t ha[4][4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    ha[kk][0] = pack_bf16(silu(z1[2 * kk][0]), silu(z1[2 * kk][1]));
    ha[kk][1] = pack_bf16(silu(z1[2 * kk][2]), silu(z1[2 * kk][3]));
    ha[kk][2] = pack_bf16(silu(z1[2 * kk + 1][0]), silu(z1[2 * kk + 1][1]));
    ha[kk][3] = pack_bf16(silu(z1[2 * kk + 1][2]), silu(z1[2 * kk + 1][3]));
  }
#pragma unroll
  for (int nn = 0; nn < 8; ++nn) {
    const float bl = S.b2[8 * nn + 2 * t], bh = S.b2[8 * nn + 2 * t + 1];
    float c[4] = {bl, bh, bl, bh};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
      mma_bf16(c, ha[kk], ld32(S.w2 + (8 * nn + g) * SW2 + 16 * kk + 2 * t),
               ld32(S.w2 + (8 * nn + g) * SW2 + 16 * kk + 2 * t + 8));
#pragma unroll
    for (int q = 0; q < 4; ++q) z2[nn][q] = c[q];
  }
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    ha[kk][0] = pack_bf16(silu(z2[2 * kk][0]), silu(z2[2 * kk][1]));
    ha[kk][1] = pack_bf16(silu(z2[2 * kk][2]), silu(z2[2 * kk][3]));
    ha[kk][2] = pack_bf16(silu(z2[2 * kk + 1][0]), silu(z2[2 * kk + 1][1]));
    ha[kk][3] = pack_bf16(silu(z2[2 * kk + 1][2]), silu(z2[2 * kk + 1][3]));
  }
  // layer 3: N = 2 padded to 8 (rows 2..7 of w3 are zero); bias on cols 0, 1
  const float bl = t == 0 ? S.b3[0] : 0.0f, bh = t == 0 ? S.b3[1] : 0.0f;
  y[0] = bl;
  y[1] = bh;
  y[2] = bl;
  y[3] = bh;
#pragma unroll
  for (int kk = 0; kk < 4; ++kk)
    mma_bf16(y, ha[kk], ld32(S.w3 + g * SW3 + 16 * kk + 2 * t), ld32(S.w3 + g * SW3 + 16 * kk + 2 * t + 8));
}

// ------------------------------------------------------------------ descriptors

struct DescConst {
  float rcut;
  int n_species;
};

__global__ void descriptor_kernel(const double *__restrict__ pos, const int32_t *__restrict__ species, int64_t n,
                                  Box B, float rcut, const int64_t *__restrict__ slice_ptr,
                                  const int32_t *__restrict__ col, const int32_t *__restrict__ cnt,
                                  const float *__restrict__ cmix, float *__restrict__ v) {
  __shared__ float sc[9 * 64];
  load_mixing(sc, cmix);
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t e0 = slice_ptr[i >> 5] + (i & 31);
  const int zi = min(max(species[i], 0), 2);
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int m = cnt[i];
  for (int s = 0; s < m; ++s) {
    const int32_t j = col[e0 + 32 * s];
    const int zj = min(max(species[j], 0), 2);
    const float r = bond_length_f32(B, pos, i, j);
    float C[8];
    bond_descriptor(r, rcut, sc + (zi * 3 + zj) * 64, C);
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] += C[k];
  }
  float4 *o = reinterpret_cast<float4 *>(v + i * 8);
  o[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
  o[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
}

// the 32 features of element e (row i, neighbour j); zeros for padding
__device__ __forceinline__ void edge_features(const double *__restrict__ pos, const int32_t *__restrict__ species,
                                              const Box &B, float rcut, const float *sc,
                                              const float *__restrict__ v, int64_t i, int32_t j, float (&x)[32]) {
  const int zi = min(max(species[i], 0), 2), zj = min(max(species[j], 0), 2);
  const float r = bond_length_f32(B, pos, i, j);
  float C[8];
  bond_descriptor(r, rcut, sc + (zi * 3 + zj) * 64, C);
  const float4 *vi4 = reinterpret_cast<const float4 *>(v + i * 8);
  const float4 *vj4 = reinterpret_cast<const float4 *>(v + (int64_t)j * 8);
  float vi[8], vj[8];
  float4 a = __ldg(vi4), b = __ldg(vi4 + 1), c = __ldg(vj4), d = __ldg(vj4 + 1);
  vi[0] = a.x; vi[1] = a.y; vi[2] = a.z; vi[3] = a.w; vi[4] = b.x; vi[5] = b.y; vi[6] = b.z; vi[7] = b.w;
  vj[0] = c.x; vj[1] = c.y; vj[2] = c.z; vj[3] = c.w; vj[4] = d.x; vj[5] = d.y; vj[6] = d.z; vj[7] = d.w;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    x[k] = C[k];
    x[8 + k] = vi[k];
    x[16 + k] = vj[k];
    x[24 + k] = C[k] * (vi[k] + vj[k]);
  }
}

// the same features with the bond length from FP32-pair positions (r^2 as an
// FP32 pair: no FP64 instruction; the inference kernel on the tensor cores)
__device__ __forceinline__ void edge_features_pair(const BoxPair &BP, const float4 *__restrict__ ph,
                                                   const float4 *__restrict__ pl, const int32_t *__restrict__ species,
                                                   float rcut, const float *sc, const float *__restrict__ v, int64_t i,
                                                   int32_t j, float (&x)[32]) {
  const int zi = min(max(species[i], 0), 2), zj = min(max(species[j], 0), 2);
  const float2 r2 = bond_r2_pair(BP, ph, pl, i, j);
  const float r = sqrtf(r2.x + r2.y);
  float C[8];
  bond_descriptor(r, rcut, sc + (zi * 3 + zj) * 64, C);
  const float4 *vi4 = reinterpret_cast<const float4 *>(v + i * 8);
  const float4 *vj4 = reinterpret_cast<const float4 *>(v + (int64_t)j * 8);
  float vi[8], vj[8];
  float4 a = __ldg(vi4), b = __ldg(vi4 + 1), c = __ldg(vj4), d = __ldg(vj4 + 1);
  vi[0] = a.x; vi[1] = a.y; vi[2] = a.z; vi[3] = a.w; vi[4] = b.x; vi[5] = b.y; vi[6] = b.z; vi[7] = b.w;
  vj[0] = c.x; vj[1] = c.y; vj[2] = c.z; vj[3] = c.w; vj[4] = d.x; vj[5] = d.y; vj[6] = d.z; vj[7] = d.w;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    x[k] = C[k];
    x[8 + k] = vi[k];
    x[16 + k] = vj[k];
    x[24 + k] = C[k] * (vi[k] + vj[k]);
  }
}

// raw FP32 features (and optionally normalised BF16) in SELL element order
__global__ void edge_feature_kernel(const double *__restrict__ pos, const int32_t *__restrict__ species, int64_t n,
                                    int64_t n_slices, Box B, float rcut, const int64_t *__restrict__ slice_ptr,
                                    const int32_t *__restrict__ col, const int32_t *__restrict__ cnt,
                                    const float *__restrict__ cmix, const float *__restrict__ v,
                                    const float *__restrict__ mean, const float *__restrict__ inv_std,
                                    float *__restrict__ xraw, bf16 *__restrict__ xb) {
  __shared__ float sc[9 * 64];
  load_mixing(sc, cmix);
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_slices * 32) return;
  const int64_t k = i >> 5;
  const int64_t e0 = slice_ptr[k] + (i & 31);
  const int w = static_cast<int>((slice_ptr[k + 1] - slice_ptr[k]) >> 5);
  const int m = i < n ? cnt[i] : 0;
  for (int s = 0; s < w; ++s) {
    const int64_t e = e0 + 32 * s;
    float x[32];
    if (s < m) {
      edge_features(pos, species, B, rcut, sc, v, i, col[e], x);
    } else {
#pragma unroll
      for (int f = 0; f < 32; ++f) x[f] = 0.0f;
    }
    if (xraw) {
      float4 *o = reinterpret_cast<float4 *>(xraw + e * 32);
#pragma unroll
      for (int q = 0; q < 8; ++q) o[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
    }
    if (xb) {
      uint32_t u[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        float lo = x[2 * q], hi = x[2 * q + 1];
        if (s < m && mean) {
          lo = (lo - mean[2 * q]) * inv_std[2 * q];
          hi = (hi - mean[2 * q + 1]) * inv_std[2 * q + 1];
        }
        u[q] = pack_bf16(lo, hi);
      }
      uint4 *o = reinterpret_cast<uint4 *>(xb + e * 32);
#pragma unroll
      for (int q = 0; q < 4; ++q) o[q] = make_uint4(u[4 * q], u[4 * q + 1], u[4 * q + 2], u[4 * q + 3]);
    }
  }
}

// per-feature sums over valid elements (FP64), one warp lane per feature
__global__ void feature_stats_kernel(const float *__restrict__ xraw, int64_t n, const int64_t *__restrict__ slice_ptr,
                                     const int32_t *__restrict__ cnt, double *__restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  double s1 = 0.0, s2 = 0.0, c = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * nw + warp; i < n; i += (int64_t)gridDim.x * nw) {
    const int64_t e0 = slice_ptr[i >> 5] + (i & 31);
    const int m = cnt[i];
    for (int s = 0; s < m; ++s) {
      const double x = xraw[(e0 + 32 * s) * 32 + lane];
      s1 += x;
      s2 += x * x;
    }
    c += m;
  }
  __shared__ double sh[8][3][32];
  sh[warp][0][lane] = s1;
  sh[warp][1][lane] = s2;
  sh[warp][2][lane] = c;
  __syncthreads();
  if (threadIdx.x < 32) {
    double a = 0, b = 0, cc = 0;
    for (int w = 0; w < nw; ++w) {
      a += sh[w][0][lane];
      b += sh[w][1][lane];
      cc += sh[w][2][lane];
    }
    part[((int64_t)blockIdx.x * 3 + 0) * 32 + lane] = a;
    part[((int64_t)blockIdx.x * 3 + 1) * 32 + lane] = b;
    part[((int64_t)blockIdx.x * 3 + 2) * 32 + lane] = cc;
  }
}

// inv_std[f] = mask[f] / max(std[f], kStdFloor) (mask 1 when absent): the
// normalisation factor of the network inputs; features with a zero mask
// are switched off
constexpr float kStdFloor = 1e-6f;
__global__ void inverse_std_kernel(const float *__restrict__ stdv, const float *__restrict__ mask,
                                   float *__restrict__ inv_std, int n) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n) return;
  inv_std[f] = (mask ? mask[f] : 1.0f) / fmaxf(stdv[f], kStdFloor);
}

__global__ void feature_stats_finish(const double *__restrict__ part, int grid, float *__restrict__ mean,
                                     float *__restrict__ stdv) {
  const int f = threadIdx.x;
  if (f >= 32) return;
  double a = 0, b = 0, c = 0;
  for (int k = 0; k < grid; ++k) {
    a += part[((int64_t)k * 3 + 0) * 32 + f];
    b += part[((int64_t)k * 3 + 1) * 32 + f];
    c += part[((int64_t)k * 3 + 2) * 32 + f];
  }
  const double m = c > 0 ? a / c : 0.0;
  const double var = c > 0 ? fmax(b / c - m * m, 0.0) : 0.0;
  mean[f] = static_cast<float>(m);
  stdv[f] = static_cast<float>(sqrt(var));
}

// ------------------------------------------------------------------ MLP forward

__global__ void __launch_bounds__(kThreads) mlp_forward_kernel(int64_t E, const bf16 *__restrict__ x,
                                                               const bf16 *__restrict__ wb,
                                                               const float *__restrict__ p, float *__restrict__ y) {
  __shared__ Weights S;
  __shared__ __align__(16) bf16 xs[TILE * SX];
  stage_weights(S, wb, p);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int64_t tile = blockIdx.x; tile * TILE < E; tile += gridDim.x) {
    const int64_t base = tile * TILE;
    __syncthreads();
    // 128 rows x 64 bytes: each thread copies one 16-byte chunk 4 times
    for (int q = threadIdx.x; q < TILE * 4; q += kThreads) {
      const int r = q >> 2, c = q & 3;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (base + r < E) v = __ldg(reinterpret_cast<const uint4 *>(x + (base + r) * NF) + c);
      *reinterpret_cast<uint4 *>(xs + r * SX + c * 8) = v;
    }
    __syncthreads();
#pragma unroll 1
    for (int mb = 0; mb < 2; ++mb) {
      const int rb = warp * 32 + mb * 16;
      float z1[8][4], z2[8][4], o[4];
      forward_block(S, xs, rb, z1, z2, o);
      if (t == 0) {
        const int64_t e_lo = base + rb + g, e_hi = base + rb + g + 8;
        if (e_lo < E) reinterpret_cast<float2 *>(y)[e_lo] = make_float2(o[0], o[1]);
        if (e_hi < E) reinterpret_cast<float2 *>(y)[e_hi] = make_float2(o[2], o[3]);
      }
    }
  }
}

// ------------------------------------------------------------------ MLP backward

// Every member starts on a 16-byte boundary: the x tile takes 16-byte
// stores and the BF16 tiles take 32-bit fragment loads.
struct BackSmem {
  alignas(16) Weights W;
  alignas(16) bf16 w2t[NH * SW2];         // W2 transposed: w2t[in][out]
  alignas(16) float w3f[2][NH];           // BF16-rounded W3 in FP32
  alignas(16) bf16 xs[TILE * SX];         // x tile [edge][feature]
  alignas(16) float dys[TILE][2];
  alignas(16) bf16 xT[NF * ST];           // [feature][edge]
  alignas(16) bf16 h1T[NH * ST];
  alignas(16) bf16 dz2T[NH * ST];
  alignas(16) bf16 dz1T[NH * ST];
  alignas(16) float bsum[4][2 * NH];      // per-warp running sums: db1 | db2
  alignas(16) float w3sum[4][2 * NH];     // per-warp running sums of dW3
  alignas(16) float db3[2];
};
static_assert(offsetof(BackSmem, xs) % 16 == 0, "x tile must be 16-byte aligned");
static_assert(offsetof(BackSmem, w2t) % 16 == 0 && offsetof(BackSmem, xT) % 16 == 0, "tile alignment");
static_assert(sizeof(BackSmem) <= 227 * 1024, "shared memory budget");

__global__ void __launch_bounds__(kThreads, 1) mlp_backward_kernel(int64_t E, const bf16 *__restrict__ x,
                                                                   const bf16 *__restrict__ wb,
                                                                   const float *__restrict__ p,
                                                                   const float *__restrict__ dy,
                                                                   float *__restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BackSmem &S = *reinterpret_cast<BackSmem *>(smem_raw);
  stage_weights(S.W, wb, p);
  for (int k = threadIdx.x; k < NH * NH; k += kThreads) S.w2t[(k % NH) * SW2 + k / NH] = wb[WB_W2 + k];
  for (int k = threadIdx.x; k < 2 * NH; k += kThreads) S.w3f[k / NH][k % NH] = __bfloat162float(wb[WB_W3 + k]);
  for (int k = threadIdx.x; k < 4 * 2 * NH; k += kThreads) {
    (&S.bsum[0][0])[k] = 0.0f;
    (&S.w3sum[0][0])[k] = 0.0f;
  }
  if (threadIdx.x < 2) S.db3[threadIdx.x] = 0.0f;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc2[8][4], acc1[4][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc2[a][b] = 0.0f;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc1[a][b] = 0.0f;

  for (int64_t tile = blockIdx.x; tile * TILE < E; tile += gridDim.x) {
    const int64_t base = tile * TILE;
    __syncthreads();
    for (int q = threadIdx.x; q < TILE * 4; q += kThreads) {
      const int r = q >> 2, c = q & 3;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (base + r < E) v = __ldg(reinterpret_cast<const uint4 *>(x + (base + r) * NF) + c);
      *reinterpret_cast<uint4 *>(S.xs + r * SX + c * 8) = v;
    }
    for (int q = threadIdx.x; q < TILE; q += kThreads) {
      float2 d = make_float2(0.0f, 0.0f);
      if (base + q < E) d = reinterpret_cast<const float2 *>(dy)[base + q];
      S.dys[q][0] = d.x;
      S.dys[q][1] = d.y;
    }
    __syncthreads();
    // ---- phase A: per 16-row block, recompute forward, form dz2 and dz1
#pragma unroll 1
    for (int mb = 0; mb < 2; ++mb) {
      const int rb = warp * 32 + mb * 16;
      float z1[8][4], z2[8][4], o[4];
      forward_block(S.W, S.xs, rb, z1, z2, o);
      const float d0g = S.dys[rb + g][0], d1g = S.dys[rb + g][1];
      const float d0h = S.dys[rb + g + 8][0], d1h = S.dys[rb + g + 8][1];
      float dz2[8][4];
#pragma unroll
      for (int nn = 0; nn < 8; ++nn)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int c = 8 * nn + 2 * t + q;
          const float w0 = S.w3f[0][c], w1 = S.w3f[1][c];
          // dW3 partial from this thread's two rows, h2 = silu(z2)
          const float h2g = silu(z2[nn][q]), h2h = silu(z2[nn][2 + q]);
          float s0 = d0g * h2g + d0h * h2h;
          float s1 = d1g * h2g + d1h * h2h;
          dz2[nn][q] = (d0g * w0 + d1g * w1) * dsilu(z2[nn][q]);
          dz2[nn][2 + q] = (d0h * w0 + d1h * w1) * dsilu(z2[nn][2 + q]);
#pragma unroll
          for (int off = 4; off < 32; off <<= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, off);
            s1 += __shfl_xor_sync(0xffffffffu, s1, off);
          }
          if (g == 0) {
            S.w3sum[warp][c] += s0;
            S.w3sum[warp][NH + c] += s1;
          }
        }
      // dh1 = dz2 W2 (B operand from W2 transposed), dz1 = dh1 * silu'(z1)
      uint32_t da[4][4];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        da[kk][0] = pack_bf16(dz2[2 * kk][0], dz2[2 * kk][1]);
        da[kk][1] = pack_bf16(dz2[2 * kk][2], dz2[2 * kk][3]);
        da[kk][2] = pack_bf16(dz2[2 * kk + 1][0], dz2[2 * kk + 1][1]);
        da[kk][3] = pack_bf16(dz2[2 * kk + 1][2], dz2[2 * kk + 1][3]);
      }
      float dz1[8][4];
#pragma unroll
      for (int nn = 0; nn < 8; ++nn) {
        float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_bf16(c, da[kk], ld32(S.w2t + (8 * nn + g) * SW2 + 16 * kk + 2 * t),
                   ld32(S.w2t + (8 * nn + g) * SW2 + 16 * kk + 2 * t + 8));
#pragma unroll
        for (int q = 0; q < 4; ++q) dz1[nn][q] = c[q] * dsilu(z1[nn][q]);
      }
      // transposed BF16 tiles for the weight-gradient MMAs, bias sums
      const int eg = rb + g, eh = rb + g + 8;
#pragma unroll
      for (int nn = 0; nn < 8; ++nn)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int c = 8 * nn + 2 * t + q;
          S.h1T[c * ST + eg] = __float2bfloat16(silu(z1[nn][q]));
          S.h1T[c * ST + eh] = __float2bfloat16(silu(z1[nn][2 + q]));
          S.dz2T[c * ST + eg] = __float2bfloat16(dz2[nn][q]);
          S.dz2T[c * ST + eh] = __float2bfloat16(dz2[nn][2 + q]);
          S.dz1T[c * ST + eg] = __float2bfloat16(dz1[nn][q]);
          S.dz1T[c * ST + eh] = __float2bfloat16(dz1[nn][2 + q]);
          float a1 = dz1[nn][q] + dz1[nn][2 + q];
          float a2 = dz2[nn][q] + dz2[nn][2 + q];
#pragma unroll
          for (int off = 4; off < 32; off <<= 1) {
            a1 += __shfl_xor_sync(0xffffffffu, a1, off);
            a2 += __shfl_xor_sync(0xffffffffu, a2, off);
          }
          if (g == 0) {
            S.bsum[warp][c] += a1;
            S.bsum[warp][NH + c] += a2;
          }
        }
      // x transposed (the 16 rows of this block, all 32 features)
#pragma unroll
      for (int kk = 0; kk < 2; ++kk)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int f0 = 16 * kk + 2 * t + q, f1 = f0 + 8;
          S.xT[f0 * ST + eg] = S.xs[eg * SX + f0];
          S.xT[f0 * ST + eh] = S.xs[eh * SX + f0];
          S.xT[f1 * ST + eg] = S.xs[eg * SX + f1];
          S.xT[f1 * ST + eh] = S.xs[eh * SX + f1];
        }
    }
    __syncthreads();
    // ---- phase B: weight gradients with the tile's 128 edges as K
    // warp w owns output rows 16w..16w+15 of dW2 (64 cols) and dW1 (32 cols)
#pragma unroll 1
    for (int kk = 0; kk < TILE / 16; ++kk) {
      uint32_t a2[4], a1[4];
      const int r0 = 16 * warp + g, r1 = r0 + 8, k0 = 16 * kk + 2 * t;
      a2[0] = ld32(S.dz2T + r0 * ST + k0);
      a2[1] = ld32(S.dz2T + r1 * ST + k0);
      a2[2] = ld32(S.dz2T + r0 * ST + k0 + 8);
      a2[3] = ld32(S.dz2T + r1 * ST + k0 + 8);
      a1[0] = ld32(S.dz1T + r0 * ST + k0);
      a1[1] = ld32(S.dz1T + r1 * ST + k0);
      a1[2] = ld32(S.dz1T + r0 * ST + k0 + 8);
      a1[3] = ld32(S.dz1T + r1 * ST + k0 + 8);
#pragma unroll
      for (int nn = 0; nn < 8; ++nn)
        mma_bf16(acc2[nn], a2, ld32(S.h1T + (8 * nn + g) * ST + k0), ld32(S.h1T + (8 * nn + g) * ST + k0 + 8));
#pragma unroll
      for (int nn = 0; nn < 4; ++nn)
        mma_bf16(acc1[nn], a1, ld32(S.xT + (8 * nn + g) * ST + k0), ld32(S.xT + (8 * nn + g) * ST + k0 + 8));
    }
    if (threadIdx.x < 2) {
      float s = 0.0f;
      for (int q = 0; q < TILE; ++q) s += S.dys[q][threadIdx.x];
      S.db3[threadIdx.x] += s;
    }
  }
  __syncthreads();
  float *out = partial + (int64_t)blockIdx.x * NPARAM;
#pragma unroll
  for (int nn = 0; nn < 8; ++nn)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int c = 8 * nn + 2 * t + q;
      out[OFF_W2 + (16 * warp + g) * NH + c] = acc2[nn][q];
      out[OFF_W2 + (16 * warp + g + 8) * NH + c] = acc2[nn][2 + q];
    }
#pragma unroll
  for (int nn = 0; nn < 4; ++nn)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int c = 8 * nn + 2 * t + q;
      out[OFF_W1 + (16 * warp + g) * NF + c] = acc1[nn][q];
      out[OFF_W1 + (16 * warp + g + 8) * NF + c] = acc1[nn][2 + q];
    }
  for (int k = threadIdx.x; k < 2 * NH; k += kThreads) {
    const float b = S.bsum[0][k] + S.bsum[1][k] + S.bsum[2][k] + S.bsum[3][k];
    out[(k < NH ? OFF_B1 : OFF_B2 - NH) + k] = b;
    out[OFF_W3 + k] = S.w3sum[0][k] + S.w3sum[1][k] + S.w3sum[2][k] + S.w3sum[3][k];
  }
  if (threadIdx.x < 2) out[OFF_B3 + threadIdx.x] = S.db3[threadIdx.x];
}

__global__ void grad_reduce_kernel(const float *__restrict__ partial, int grid, float *__restrict__ grad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NPARAM) return;
  double s = 0.0;
  for (int c = 0; c < grid; ++c) s += partial[(int64_t)c * NPARAM + k];
  grad[k] = static_cast<float>(s);
}

// ------------------------------------------------------------------ loss (Eq. 3 form)

// pass 1: residual sums over the rows [r0, r1): |D|, D^2 and the count
__global__ void loss_sums_kernel(int64_t r0, int64_t r1, const int64_t *__restrict__ slice_ptr,
                                 const int32_t *__restrict__ cnt, const float *__restrict__ y,
                                 const float *__restrict__ t_hop, const float *__restrict__ eps_t,
                                 const int32_t *__restrict__ species, const float *__restrict__ eps0,
                                 double *__restrict__ part) {
  double sa = 0.0, sq = 0.0, c = 0.0;
  for (int64_t i = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r1;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e0 = slice_ptr[i >> 5] + (i & 31);
    const int m = cnt[i];
    double eps = eps0[min(max(species[i], 0), 2)];
    for (int s = 0; s < m; ++s) {
      const int64_t e = e0 + 32 * s;
      const double d = (double)y[2 * e] - (double)t_hop[e];
      sa += fabs(d);
      sq += d * d;
      eps += (double)y[2 * e + 1];
    }
    const double don = eps - (double)eps_t[i];
    sa += fabs(don);
    sq += don * don;
    c += m + 1;
  }
  __shared__ double sh[3][32];
  for (int off = 16; off > 0; off >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, off);
    sq += __shfl_xor_sync(0xffffffffu, sq, off);
    c += __shfl_xor_sync(0xffffffffu, c, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][warp] = sa;
    sh[1][warp] = sq;
    sh[2][warp] = c;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[threadIdx.x][w];
    part[(int64_t)blockIdx.x * 3 + threadIdx.x] = s;
  }
}

// stats[0..2] = sum|D|/n, sum D^2/n, n; stats[3] = loss
__global__ void loss_finish_kernel(const double *__restrict__ part, int grid, double *__restrict__ stats) {
  if (threadIdx.x != 0) return;
  double a = 0, b = 0, c = 0;
  for (int k = 0; k < grid; ++k) {
    a += part[3 * k];
    b += part[3 * k + 1];
    c += part[3 * k + 2];
  }
  const double n = c > 0 ? c : 1.0;
  stats[0] = a / n;
  stats[1] = b / n;
  stats[2] = c;
  stats[3] = (a / n) * (a / n) + b / n;
}

__device__ __forceinline__ double sgn(double d) { return d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0); }

// pass 2: dL/dy for every element of the rows (padding slots get 0)
__global__ void loss_grad_kernel(int64_t r0, int64_t r1, const int64_t *__restrict__ slice_ptr,
                                 const int32_t *__restrict__ cnt, const float *__restrict__ y,
                                 const float *__restrict__ t_hop, const float *__restrict__ eps_t,
                                 const int32_t *__restrict__ species, const float *__restrict__ eps0,
                                 const double *__restrict__ stats, float *__restrict__ dy) {
  const int64_t i = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= r1) return;
  const double sabs = stats[0], n = stats[2] > 0 ? stats[2] : 1.0;
  const int64_t k = i >> 5;
  const int64_t e0 = slice_ptr[k] + (i & 31);
  const int w = static_cast<int>((slice_ptr[k + 1] - slice_ptr[k]) >> 5);
  const int m = cnt[i];
  double eps = eps0[min(max(species[i], 0), 2)];
  for (int s = 0; s < m; ++s) eps += (double)y[2 * (e0 + 32 * s) + 1];
  const double don = eps - (double)eps_t[i];
  const double g_on = 2.0 * sabs * sgn(don) / n + 2.0 * don / n;
  for (int s = 0; s < w; ++s) {
    const int64_t e = e0 + 32 * s;
    float2 o = make_float2(0.0f, 0.0f);
    if (s < m) {
      const double d = (double)y[2 * e] - (double)t_hop[e];
      o.x = static_cast<float>(2.0 * sabs * sgn(d) / n + 2.0 * d / n);
      o.y = static_cast<float>(g_on);
    }
    reinterpret_cast<float2 *>(dy)[e] = o;
  }
}

// ------------------------------------------------------------------ AdamW

__global__ void adamw_kernel(float *__restrict__ p, const float *__restrict__ grad, float *__restrict__ m,
                             float *__restrict__ v, int64_t step, float lr, float beta1, float beta2, float eps,
                             float wd, bf16 *__restrict__ wb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NPARAM) return;
  const float g = grad[k];
  float pk = p[k] * (1.0f - lr * wd);
  const float mk = beta1 * m[k] + (1.0f - beta1) * g;
  const float vk = beta2 * v[k] + (1.0f - beta2) * g * g;
  const double bc1 = 1.0 - pow((double)beta1, (double)step);
  const double bc2 = 1.0 - pow((double)beta2, (double)step);
  const float mhat = static_cast<float>(mk / bc1);
  const float vhat = static_cast<float>(vk / bc2);
  pk -= lr * mhat / (sqrtf(vhat) + eps);
  p[k] = pk;
  m[k] = mk;
  v[k] = vk;
  int wi = -1;
  if (k < OFF_B1) wi = WB_W1 + k;
  else if (k >= OFF_W2 && k < OFF_B2) wi = WB_W2 + (k - OFF_W2);
  else if (k >= OFF_W3 && k < OFF_B3) wi = WB_W3 + (k - OFF_W3);
  if (wi >= 0) wb[wi] = __float2bfloat16(pk);
}

__global__ void pack_weights_kernel(const float *__restrict__ p, bf16 *__restrict__ wb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NPARAM) return;
  int wi = -1;
  if (k < OFF_B1) wi = WB_W1 + k;
  else if (k >= OFF_W2 && k < OFF_B2) wi = WB_W2 + (k - OFF_W2);
  else if (k >= OFF_W3 && k < OFF_B3) wi = WB_W3 + (k - OFF_W3);
  if (wi >= 0) wb[wi] = __float2bfloat16(p[k]);
}

// ------------------------------------------------------------------ learned H

// per slice: features -> MLP -> y0 (hopping, directed) and y1 (onsite share)
__global__ void __launch_bounds__(kThreads) mlp_hamiltonian_kernel(
    const double *__restrict__ pos, const int32_t *__restrict__ species, int64_t n, int64_t n_slices, Box B,
    float rcut, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ col,
    const int32_t *__restrict__ cnt, const float *__restrict__ cmix, const float *__restrict__ v,
    const float *__restrict__ mean, const float *__restrict__ inv_std, const bf16 *__restrict__ wb,
    const float *__restrict__ p, float *__restrict__ y0, float *__restrict__ y1) {
  __shared__ Weights S;
  __shared__ float sc[9 * 64];
  __shared__ float smean[32], sinv[32];
  __shared__ __align__(16) bf16 xs[TILE * SX];
  stage_weights(S, wb, p);
  load_mixing(sc, cmix);
  if (threadIdx.x < 32) {
    smean[threadIdx.x] = mean ? mean[threadIdx.x] : 0.0f;
    sinv[threadIdx.x] = inv_std ? inv_std[threadIdx.x] : 1.0f;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int64_t k = blockIdx.x; k < n_slices; k += gridDim.x) {
    const int64_t sb = slice_ptr[k];
    const int w = static_cast<int>((slice_ptr[k + 1] - sb) >> 5);
    for (int c0 = 0; c0 < w; c0 += 4) {
      __syncthreads();
      {  // features of element q = threadIdx.x: slot c0 + warp, lane
        const int slot = c0 + warp;
        const int64_t i = k * 32 + lane;
        float x[32];
        const bool valid = slot < w && i < n && slot < cnt[i];
        if (valid) {
          edge_features(pos, species, B, rcut, sc, v, i, col[sb + 32 * slot + lane], x);
#pragma unroll
          for (int f = 0; f < 32; ++f) x[f] = (x[f] - smean[f]) * sinv[f];
        } else {
#pragma unroll
          for (int f = 0; f < 32; ++f) x[f] = 0.0f;
        }
        uint32_t u[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) u[q] = pack_bf16(x[2 * q], x[2 * q + 1]);
        uint4 *o = reinterpret_cast<uint4 *>(xs + threadIdx.x * SX);
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = make_uint4(u[4 * q], u[4 * q + 1], u[4 * q + 2], u[4 * q + 3]);
      }
      __syncthreads();
#pragma unroll 1
      for (int mb = 0; mb < 2; ++mb) {
        const int rb = warp * 32 + mb * 16;
        float z1[8][4], z2[8][4], o[4];
        forward_block(S, xs, rb, z1, z2, o);
        if (t == 0) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int q = rb + g + 8 * h;  // tile row = element index in chunk
            const int slot = c0 + (q >> 5);
            const int64_t i = k * 32 + (q & 31);
            if (slot < w && i < n && slot < cnt[i]) {
              const int64_t e = sb + 32 * slot + (q & 31);
              y0[e] = o[2 * h];
              y1[e] = o[2 * h + 1];
            }
          }
        }
      }
    }
  }
}

// The same forward pass on the 5th-generation tensor cores (tcgen05).  A CTA
// of 4 warps owns a tile of 128 edges = the 128 TMEM lanes; thread t builds
// edge t's features and owns row t of every accumulator.  Per tile:
//   X (128 x 32, BF16, shared) . W1^T -> D1 (TMEM cols 0..63)      2 MMAs (K = 16)
//   silu(D1 + b1) -> H (shared, the A operand of the next layer)
//   H . W2^T -> D2 (cols 64..127)                                   4 MMAs
//   silu(D2 + b2) -> H;  H . W3^T -> D3 (cols 0..15, W3 padded)     4 MMAs
//   y = D3[:, 0:2] + b3
// One thread issues each layer's MMAs and commits them to an mbarrier that
// every thread waits on (bounded: on timeout the CTA raises flags[0] |= 2,
// waits once more for its MMAs, frees its TMEM and stops).  Operands use the
// K-major core-matrix layout without swizzle; the weights stay in shared
// memory for the whole kernel.  128 TMEM columns per CTA; the dynamic
// shared-memory request keeps at most 4 CTAs (512 columns) on an SM.
struct TcSmem {
  bf16 w1[64 * 32];
  bf16 w2[64 * 64];
  bf16 w3[16 * 64];
  bf16 xa[TILE * 32];
  bf16 ha[TILE * 64];
  float b1[64], b2[64], b3[2];
  float sc[9 * 64];
  float smean[32], sinv[32];
  uint64_t bar;
  uint32_t tmem;
};
// kernel of the learned-H forward: 0 = tcgen05 (default), 1 = mma.sync
int g_mlp_variant = 0;

constexpr size_t kTcSmemBytes = sizeof(TcSmem) + 128 > 47 * 1024 ? sizeof(TcSmem) + 128 : 47 * 1024;
constexpr long long kTcPolls = 1ll << 22;

__device__ __forceinline__ void store_row8(bf16 *tile, int row, int k0, int kdim, const float (&v)[8]) {
  uint4 u = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
  *reinterpret_cast<uint4 *>(tile + tc::core_index(row, k0, kdim)) = u;
}

// every thread: all of this CTA's MMAs issued so far have completed?
__device__ __forceinline__ bool tc_layer_wait(TcSmem &S, uint32_t &phase, int *flags) {
  const bool ok = __syncthreads_and(tc::mbar_wait(&S.bar, phase, kTcPolls)) != 0;
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(flags, 2);
    tc::mbar_wait(&S.bar, phase, kTcPolls);   // drain the MMAs in flight before TMEM is freed
  }
  phase ^= 1u;
  tc::fence_after_sync();
  return ok;
}

// generic writes of the A operand done: make them visible to the tensor core
__device__ __forceinline__ void tc_operands_ready() {
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
}

__global__ void __launch_bounds__(kThreads) mlp_hamiltonian_tc_kernel(
    const float4 *__restrict__ ph, const float4 *__restrict__ pl, const int32_t *__restrict__ species, int64_t n,
    int64_t n_slices, BoxPair BP, float rcut, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ col,
    const int32_t *__restrict__ cnt, const float *__restrict__ cmix, const float *__restrict__ v,
    const float *__restrict__ mean, const float *__restrict__ inv_std, const bf16 *__restrict__ wb,
    const float *__restrict__ p, float *__restrict__ y0, float *__restrict__ y1, int *__restrict__ flags) {
  extern __shared__ __align__(128) unsigned char tc_raw[];
  TcSmem &S = *reinterpret_cast<TcSmem *>(tc_raw + ((128 - (smem_u32_generic(tc_raw) & 127)) & 127));
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int e = tid; e < 64 * 32; e += kThreads) S.w1[tc::core_index(e >> 5, e & 31, 32)] = wb[WB_W1 + e];
  for (int e = tid; e < 64 * 64; e += kThreads) S.w2[tc::core_index(e >> 6, e & 63, 64)] = wb[WB_W2 + e];
  for (int e = tid; e < 16 * 64; e += kThreads)
    S.w3[tc::core_index(e >> 6, e & 63, 64)] = (e >> 6) < 2 ? wb[WB_W3 + e] : __float2bfloat16(0.0f);
  for (int e = tid; e < 64; e += kThreads) {
    S.b1[e] = p[OFF_B1 + e];
    S.b2[e] = p[OFF_B2 + e];
  }
  if (tid < 2) S.b3[tid] = p[OFF_B3 + tid];
  load_mixing(S.sc, cmix);
  if (tid < 32) {
    S.smean[tid] = mean ? mean[tid] : 0.0f;
    S.sinv[tid] = inv_std ? inv_std[tid] : 1.0f;
  }
  if (tid == 0) tc::mbar_init(&S.bar, 1);
  if (warp == 0) tc::alloc(&S.tmem, 128);
  tc_operands_ready();
  const uint32_t tmem = S.tmem;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t id64 = tc::idesc_bf16(TILE, 64), id16 = tc::idesc_bf16(TILE, 16);
  uint32_t phase = 0;
  bool ok = true;
  for (int64_t k = blockIdx.x; k < n_slices && ok; k += gridDim.x) {
    const int64_t sb = slice_ptr[k];
    const int w = static_cast<int>((slice_ptr[k + 1] - sb) >> 5);
    for (int c0 = 0; c0 < w && ok; c0 += 4) {
      // features of edge tid: slot c0 + warp of row k*32 + lane
      const int slot = c0 + warp;
      const int64_t i = k * 32 + (tid & 31);
      const bool valid = slot < w && i < n && slot < cnt[i];
      {
        float x[32];
        if (valid) {
          edge_features_pair(BP, ph, pl, species, rcut, S.sc, v, i, col[sb + 32 * slot + (tid & 31)], x);
#pragma unroll
          for (int f = 0; f < 32; ++f) x[f] = (x[f] - S.smean[f]) * S.sinv[f];
        } else {
#pragma unroll
          for (int f = 0; f < 32; ++f) x[f] = 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float c8[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) c8[j] = x[8 * q + j];
          store_row8(S.xa, tid, 8 * q, 32, c8);
        }
      }
      tc_operands_ready();
      if (tid == 0) {
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
          tc::mma_bf16(tmem, tc::desc_kmajor(S.xa + ks * 128, 32), tc::desc_kmajor(S.w1 + ks * 128, 32), id64,
                       ks > 0);
        tc::commit(&S.bar);
      }
      if (!(ok = tc_layer_wait(S, phase, flags))) break;
      // layer 1 epilogue: H = silu(D1 + b1)
#pragma unroll 1
      for (int c = 0; c < 64; c += 16) {
        float d[16];
        tc::ld16(tmem + lane_base + (uint32_t)c, d);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float c8[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) c8[j] = silu(d[8 * h + j] + S.b1[c + 8 * h + j]);
          store_row8(S.ha, tid, c + 8 * h, 64, c8);
        }
      }
      tc_operands_ready();
      if (tid == 0) {
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          tc::mma_bf16(tmem + 64, tc::desc_kmajor(S.ha + ks * 128, 64), tc::desc_kmajor(S.w2 + ks * 128, 64), id64,
                       ks > 0);
        tc::commit(&S.bar);
      }
      if (!(ok = tc_layer_wait(S, phase, flags))) break;
      // layer 2 epilogue: H = silu(D2 + b2) (layer 2 has finished reading H)
#pragma unroll 1
      for (int c = 0; c < 64; c += 16) {
        float d[16];
        tc::ld16(tmem + lane_base + 64u + (uint32_t)c, d);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float c8[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) c8[j] = silu(d[8 * h + j] + S.b2[c + 8 * h + j]);
          store_row8(S.ha, tid, c + 8 * h, 64, c8);
        }
      }
      tc_operands_ready();
      if (tid == 0) {
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          tc::mma_bf16(tmem, tc::desc_kmajor(S.ha + ks * 128, 64), tc::desc_kmajor(S.w3 + ks * 128, 64), id16,
                       ks > 0);
        tc::commit(&S.bar);
      }
      if (!(ok = tc_layer_wait(S, phase, flags))) break;
      float o[2];
      tc::ld2(tmem + lane_base, o);
      if (valid) {
        const int64_t e = sb + 32 * slot + (tid & 31);
        y0[e] = o[0] + S.b3[0];
        y1[e] = o[1] + S.b3[1];
      }
      tc::fence_before_sync();   // D3 read before the next tile's layer 1 overwrites it
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, 128);
}

// val = (y0(i->j) + y0(j->i)) / 2, diag = eps0[Z_i] + sum_j y1(i->j)
constexpr int kAsmW = 16;   // rows of slices at most this wide search their mirrors together
template <typename valT>
__global__ void learned_assemble_kernel(int64_t n, int64_t n_slices, const int64_t *__restrict__ slice_ptr,
                                        const int32_t *__restrict__ col, const int32_t *__restrict__ cnt,
                                        const int32_t *__restrict__ species, const float *__restrict__ eps0,
                                        const float *__restrict__ y0, const float *__restrict__ y1,
                                        valT *__restrict__ val, valT *__restrict__ diag, int *__restrict__ flags) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_slices * 32) return;
  const int64_t k = i >> 5;
  const int64_t e0 = slice_ptr[k] + (i & 31);
  const int w = static_cast<int>((slice_ptr[k + 1] - slice_ptr[k]) >> 5);
  const int m = i < n ? cnt[i] : 0;
  double eps = i < n ? (double)eps0[min(max(species[i], 0), 2)] : 0.0;
  if (w <= kAsmW) {
    // the row's mirror searches advance together, one level per round, so
    // that their dependent loads overlap (same results as one at a time)
    int32_t jj[kAsmW];
    int64_t f0[kAsmW];
    int lo[kAsmW], hi[kAsmW], found[kAsmW];
#pragma unroll
    for (int s = 0; s < kAsmW; ++s) {
      found[s] = -1;
      lo[s] = 0;
      hi[s] = -1;
      if (s < m) {
        jj[s] = col[e0 + 32 * s];
        f0[s] = slice_ptr[jj[s] >> 5] + (jj[s] & 31);
        hi[s] = cnt[jj[s]] - 1;
      }
    }
    for (int round = 0; round < 32; ++round) {
      bool active = false;
#pragma unroll
      for (int s = 0; s < kAsmW; ++s) {
        if (s < m && found[s] < 0 && lo[s] <= hi[s]) {
          const int mid = (lo[s] + hi[s]) >> 1;
          const int32_t cj = col[f0[s] + 32 * mid];
          if (cj == i) found[s] = mid;
          else if (cj < i) lo[s] = mid + 1;
          else hi[s] = mid - 1;
          active = true;
        }
      }
      if (!active) break;
    }
#pragma unroll
    for (int s = 0; s < kAsmW; ++s) {
      if (s >= w) break;
      const int64_t e = e0 + 32 * s;
      double h = 0.0;
      if (s < m) {
        if (found[s] < 0) {
          atomicOr(flags, 1);
          h = y0[e];
        } else {
          h = 0.5 * ((double)y0[e] + (double)y0[f0[s] + 32 * found[s]]);
        }
        eps += (double)y1[e];
      }
      val[e] = static_cast<valT>(h);
    }
    if (i < n && diag) diag[i] = static_cast<valT>(eps);
    return;
  }
  for (int s = 0; s < w; ++s) {
    const int64_t e = e0 + 32 * s;
    double h = 0.0;
    if (s < m) {
      const int32_t j = col[e];
      // find i in row j (its neighbours are sorted ascending)
      const int64_t f0 = slice_ptr[j >> 5] + (j & 31);
      int lo = 0, hi = cnt[j] - 1, found = -1;
      while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int32_t cj = col[f0 + 32 * mid];
        if (cj == i) {
          found = mid;
          break;
        }
        if (cj < i) lo = mid + 1;
        else hi = mid - 1;
      }
      if (found < 0) {
        atomicOr(flags, 1);
        h = y0[e];
      } else {
        h = 0.5 * ((double)y0[e] + (double)y0[f0 + 32 * found]);
      }
      eps += (double)y1[e];
    }
    val[e] = static_cast<valT>(h);
  }
  if (i < n && diag) diag[i] = static_cast<valT>(eps);
}

int grid_cap(int64_t units, int per_sm) {
  const int64_t cap = (int64_t)sm_count() * per_sm;
  return static_cast<int>(units < cap ? (units > 0 ? units : 1) : cap);
}

}  // namespace
}  // namespace gputb

using namespace gputb;

// ------------------------------------------------------------------ C ABI

extern "C" tb_status tb_compute_descriptors(const double *positions, const int32_t *species, int64_t n,
                                            const double *box, const int32_t *pbc, double rcut,
                                            const int64_t *slice_ptr, const int32_t *col, const int32_t *cnt,
                                            const float *cmix, float *v, void *stream) {
  TB_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "tb_compute_descriptors: bad n");
  TB_REQUIRE(positions && species && slice_ptr && cnt && cmix && v, "tb_compute_descriptors: null pointer");
  Box B;
  tb_status s = make_box(box, pbc, rcut, &B);
  if (s != TB_OK) return s;
  descriptor_kernel<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      positions, species, n, B, (float)rcut, slice_ptr, col, cnt, cmix, v);
  TB_CHECK_LAUNCH();
  return TB_OK;
}

extern "C" tb_status tb_edge_features(const double *positions, const int32_t *species, int64_t n,
                                      const double *box, const int32_t *pbc, double rcut,
                                      const int64_t *slice_ptr, const int32_t *col, const int32_t *cnt,
                                      const float *cmix, const float *v, const float *mean, const float *inv_std,
                                      float *x_raw, void *x_bf16, void *stream) {
  TB_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "tb_edge_features: bad n");
  TB_REQUIRE(positions && species && slice_ptr && cnt && cmix && v, "tb_edge_features: null pointer");
  TB_REQUIRE(x_raw || x_bf16, "tb_edge_features: no output requested");
  TB_REQUIRE((mean == nullptr) == (inv_std == nullptr), "tb_edge_features: mean and inv_std go together");
  Box B;
  tb_status s = make_box(box, pbc, rcut, &B);
  if (s != TB_OK) return s;
  const int64_t n_slices = (n + 31) / 32;
  edge_feature_kernel<<<(unsigned)((n_slices * 32 + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
      positions, species, n, n_slices, B, (float)rcut, slice_ptr, col, cnt, cmix, v, mean, inv_std, x_raw,
      static_cast<bf16 *>(x_bf16));
  TB_CHECK_LAUNCH();
  return TB_OK;
}

extern "C" tb_status tb_feature_stats(const float *x_raw, int64_t n, const int64_t *slice_ptr, const int32_t *cnt,
                                      float *mean, float *stdv, float *inv_std, const float *mask, void *workspace,
                                      size_t workspace_bytes, void *stream) {
  TB_REQUIRE(n >= 1 && x_raw && slice_ptr && cnt && mean && stdv && workspace, "tb_feature_stats: bad argument");
  const int grid = grid_cap((n + 7) / 8, 4);
  if (workspace_bytes < (size_t)grid * 96 * sizeof(double))
    return fail(TB_ERR_WORKSPACE, "tb_feature_stats: workspace needs %zu bytes", (size_t)grid * 96 * 8);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double *part = static_cast<double *>(workspace);
  feature_stats_kernel<<<grid, 256, 0, st>>>(x_raw, n, slice_ptr, cnt, part);
  TB_CHECK_LAUNCH();
  feature_stats_finish<<<1, 32, 0, st>>>(part, grid, mean, stdv);
  TB_CHECK_LAUNCH();
  if (inv_std) {
    inverse_std_kernel<<<1, 32, 0, st>>>(stdv, mask, inv_std, 32);
    TB_CHECK_LAUNCH();
  }
  return TB_OK;
}

extern "C" tb_status tb_inverse_std(const float *stdv, const float *mask, float *inv_std, int32_t n, void *stream) {
  TB_REQUIRE(n >= 1 && n <= (1 << 20) && stdv && inv_std, "tb_inverse_std: bad argument");
  inverse_std_kernel<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(stdv, mask, inv_std, n);
  TB_CHECK_LAUNCH();
  return TB_OK;
}

extern "C" size_t tb_mlp_workspace_size(int64_t n_edges) {
  if (n_edges < 0) return 0;
  const int grid = grid_cap((n_edges + TILE - 1) / TILE, 1);
  return align_up((size_t)grid * NPARAM * sizeof(float), 256) + align_up(4096 * sizeof(double), 256) + 256;
}

extern "C" tb_status tb_mlp_forward(int64_t n_edges, const void *x_bf16, const void *w_bf16, const float *params,
                                    float *y, void *stream) {
  TB_REQUIRE(n_edges >= 0 && (n_edges == 0 || (x_bf16 && w_bf16 && params && y)), "tb_mlp_forward: bad argument");
  if (n_edges == 0) return TB_OK;
  const int grid = grid_cap((n_edges + TILE - 1) / TILE, 8);
  mlp_forward_kernel<<<grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      n_edges, static_cast<const bf16 *>(x_bf16), static_cast<const bf16 *>(w_bf16), params, y);
  TB_CHECK_LAUNCH();
  return TB_OK;
}

extern "C" tb_status tb_mlp_backward(int64_t n_edges, const void *x_bf16, const void *w_bf16, const float *params,
                                     const float *dy, float *grad, void *workspace, size_t workspace_bytes,
                                     void *stream) {
  TB_REQUIRE(n_edges >= 1 && x_bf16 && w_bf16 && params && dy && grad && workspace, "tb_mlp_backward: bad argument");
  const int grid = grid_cap((n_edges + TILE - 1) / TILE, 1);
  if (workspace_bytes < tb_mlp_workspace_size(n_edges))
    return fail(TB_ERR_WORKSPACE, "tb_mlp_backward: workspace too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t smem = sizeof(BackSmem);
  TB_CUDA(cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  float *partial = static_cast<float *>(workspace);
  mlp_backward_kernel<<<grid, kThreads, smem, st>>>(n_edges, static_cast<const bf16 *>(x_bf16),
                                                    static_cast<const bf16 *>(w_bf16), params, dy, partial);
  TB_CHECK_LAUNCH();
  grad_reduce_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(partial, grid, grad);
  TB_CHECK_LAUNCH();
  return TB_OK;
}

extern "C" tb_status tb_mlp_loss(int64_t row_begin, int64_t row_end, const int64_t *slice_ptr, const int32_t *cnt,
                                 const float *y, const float *t_hop, const float *eps_target,
                                 const int32_t *species, const float *eps0, float *dy, double *stats,
                                 void *workspace, size_t workspace_bytes, void *stream) {
  TB_REQUIRE(row_end > row_begin && row_begin >= 0, "tb_mlp_loss: empty row range");
  TB_REQUIRE(slice_ptr && cnt && y && t_hop && eps_target && species && eps0 && dy && stats && workspace,
             "tb_mlp_loss: null pointer");
  const int64_t rows = row_end - row_begin;
  const int grid = grid_cap((rows + 255) / 256, 2);
  if (workspace_bytes < (size_t)grid * 3 * sizeof(double))
    return fail(TB_ERR_WORKSPACE, "tb_mlp_loss: workspace too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double *part = static_cast<double *>(workspace);
  loss_sums_kernel<<<grid, 256, 0, st>>>(row_begin, row_end, slice_ptr, cnt, y, t_hop, eps_target, species, eps0,
                                         part);
  TB_CHECK_LAUNCH();
  loss_finish_kernel<<<1, 32, 0, st>>>(part, grid, stats);
  TB_CHECK_LAUNCH();
  loss_grad_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(row_begin, row_end, slice_ptr, cnt, y, t_hop,
                                                                    eps_target, species, eps0, stats, dy);
  TB_CHECK_LAUNCH();
  return TB_OK;
}

extern "C" tb_status tb_adamw_step(float *params, const float *grad, float *m, float *v, int64_t step, double lr,
                                   double beta1, double beta2, double eps, double weight_decay, void *w_bf16,
                                   void *stream) {
  TB_REQUIRE(params && grad && m && v && w_bf16 && step >= 1, "tb_adamw_step: bad argument");
  adamw_kernel<<<(NPARAM + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      params, grad, m, v, step, (float)lr, (float)beta1, (float)beta2, (float)eps, (float)weight_decay,
      static_cast<bf16 *>(w_bf16));
  TB_CHECK_LAUNCH();
  return TB_OK;
}

extern "C" tb_status tb_mlp_pack_weights(const float *params, void *w_bf16, void *stream) {
  TB_REQUIRE(params && w_bf16, "tb_mlp_pack_weights: null pointer");
  pack_weights_kernel<<<(NPARAM + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      params, static_cast<bf16 *>(w_bf16));
  TB_CHECK_LAUNCH();
  return TB_OK;
}

extern "C" size_t tb_build_hamiltonian_workspace_size(int64_t n, int64_t total_elements) {
  if (n < 0 || total_elements < 0) return 0;
  // y0 and y1 per element, the status words, the FP32-pair positions
  return 2 * align_up((size_t)(total_elements > 0 ? total_elements : 1) * sizeof(float), 256) + 512 +
         2 * align_up((size_t)n * sizeof(float4), 256);
}

extern "C" tb_status tb_build_hamiltonian(const double *positions, const int32_t *species, int64_t n,
                                          const double *box, const int32_t *pbc, double rcut,
                                          const int64_t *slice_ptr, const int32_t *col, const int32_t *cnt,
                                          int64_t total_elements, const float *cmix, const float *v,
                                          const float *mean, const float *inv_std, const void *w_bf16,
                                          const float *params, const float *eps0, int32_t precision, void *val,
                                          void *diag, void *workspace, size_t workspace_bytes, void *stream) {
  TB_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "tb_build_hamiltonian: bad n");
  TB_REQUIRE(positions && species && slice_ptr && cnt && cmix && v && w_bf16 && params && eps0 && workspace,
             "tb_build_hamiltonian: null pointer");
  TB_REQUIRE(total_elements == 0 || (col && val), "tb_build_hamiltonian: col and val are required");
  TB_REQUIRE(precision == TB_F32 || precision == TB_F64, "tb_build_hamiltonian: bad precision");
  if (workspace_bytes < tb_build_hamiltonian_workspace_size(n, total_elements))
    return fail(TB_ERR_WORKSPACE, "tb_build_hamiltonian: workspace too small");
  Box B;
  tb_status s = make_box(box, pbc, rcut, &B);
  if (s != TB_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carver cv(workspace, workspace_bytes);
  float *y0 = cv.take<float>(total_elements > 0 ? total_elements : 1);
  float *y1 = cv.take<float>(total_elements > 0 ? total_elements : 1);
  int *flags = cv.take<int>(4);
  float4 *ph = cv.take<float4>(n), *pl = cv.take<float4>(n);
  TB_CUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
  const int64_t n_slices = (n + 31) / 32;
  if (g_mlp_variant == 1) {
    const int grid = grid_cap(n_slices, 8);
    mlp_hamiltonian_kernel<<<grid, kThreads, 0, st>>>(positions, species, n, n_slices, B, (float)rcut, slice_ptr,
                                                      col, cnt, cmix, v, mean, inv_std,
                                                      static_cast<const bf16 *>(w_bf16), params, y0, y1);
  } else {
    pos_pair_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(positions, n, ph, pl);
    TB_CHECK_LAUNCH();
    const int grid = grid_cap(n_slices, 4);
    mlp_hamiltonian_tc_kernel<<<grid, kThreads, kTcSmemBytes, st>>>(
        ph, pl, species, n, n_slices, box_pair(B), (float)rcut, slice_ptr, col, cnt, cmix, v, mean, inv_std,
        static_cast<const bf16 *>(w_bf16), params, y0, y1, flags);
  }
  TB_CHECK_LAUNCH();
  const unsigned nb = (unsigned)((n_slices * 32 + 255) / 256);
  if (precision == TB_F32)
    learned_assemble_kernel<float><<<nb, 256, 0, st>>>(n, n_slices, slice_ptr, col, cnt, species, eps0, y0, y1,
                                                       static_cast<float *>(val), static_cast<float *>(diag), flags);
  else
    learned_assemble_kernel<double><<<nb, 256, 0, st>>>(n, n_slices, slice_ptr, col, cnt, species, eps0, y0, y1,
                                                        static_cast<double *>(val), static_cast<double *>(diag),
                                                        flags);
  TB_CHECK_LAUNCH();
  int h = 0;
  TB_CUDA(cudaMemcpyAsync(&h, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  TB_CUDA(cudaStreamSynchronize(st));
  if (h & 2) return fail(TB_ERR_TIMEOUT, "tb_build_hamiltonian: a tensor-core completion wait timed out");
  if (h & 1) return fail(TB_ERR_INVALID_ARG, "tb_build_hamiltonian: neighbour relation is not symmetric");
  return TB_OK;
}

extern "C" tb_status tb_mlp_set_variant(int32_t variant) {
  TB_REQUIRE(variant == 0 || variant == 1, "tb_mlp_set_variant: variant must be 0 (tcgen05) or 1 (mma.sync)");
  g_mlp_variant = variant;
  return TB_OK;
}
