// Environment-network model and band-energy training (Eq. 2 edge feature,
// the SK form of the hopping and the onsite network of Sec. 3, the band loss
// of Eq. 3):
//
//   u_ij = v_i + v_j,  m = MLP_e(u) (8-32-8),  e_ij = C(r_ij) * m,
//   y = MLP_lambda(e) (8-32-32-2),  t_ij = y_sigma n_z^2 + y_pi (1 - n_z^2),
//   eps_i = eps0[Z_i] + MLP_alpha(v_i)[Z_i] (8-32-3),
//   H(k)_ij = sum over stored (i, j, d) of t e^{i k.d} + eps_i delta_ij,
//   bands = eigenvalues of H(k),  L = (sum w_b |D|)^2 + sum w_b D^2.
//
// The networks are a few thousand FP32 operations per bond with widths of
// 8 and 32, so they run on the FP32 pipes with the weights in shared memory
// (a warp reads one weight at a time: broadcast).  Bloch matrices are at
// most 64 x 64: one CTA builds H(k) in shared memory and diagonalises it by
// cyclic Jacobi rotations in the round-robin order (n/2 disjoint rotations
// per round, applied by all threads), so a whole batch of cells and k-points
// is one launch with no host round trip.  Gradients: Hellmann-Feynman for
// the bands, then the networks' backward pass with per-CTA partial sums
// reduced in a fixed order (reproducible).
#include <cmath>
#include <cstddef>
#include <cstring>

#include <cuda_bf16.h>

#include "common.cuh"
#include "descriptor.cuh"
#include "geometry.cuh"
#include "tcgen05.cuh"

namespace gputb {
namespace {

// flat parameter layout (weights [out][in] row-major, then biases)
constexpr int oWe1 = 0, obe1 = 256, oWe2 = 288, obe2 = 544;
constexpr int oWh1 = 552, obh1 = 808, oWh2 = 840, obh2 = 1864, oWh3 = 1896, obh3 = 1960;
constexpr int oWo1 = 1962, obo1 = 2218, oWo2 = 2250, obo2 = 2346;
constexpr int kNP = TB_ENV_NPARAM;
static_assert(obo2 + 3 == kNP, "parameter layout");
constexpr int kNF = TB_ENV_NFEAT;  // C[8], u[8], n_z^2, d[3]
constexpr int kMaxBand = 64;
constexpr int kMaxCnt = 32;

// onsite block shifted by two floats in shared memory so that every weight
// row starts on a 16-byte boundary (float4 broadcast loads)
constexpr int kShift = 2;
constexpr int sWo1 = oWo1 + kShift, sbo1 = obo1 + kShift, sWo2 = oWo2 + kShift, sbo2 = obo2 + kShift;
constexpr int kNPs = kNP + kShift;
static_assert(oWe2 % 4 == 0 && oWh1 % 4 == 0 && oWh2 % 4 == 0 && oWh3 % 4 == 0 && sWo1 % 4 == 0 && sWo2 % 4 == 0,
              "weight rows 16-byte aligned in shared memory");

// logistic function from the hardware exponential and divide (a few ulp;
// the argument is clamped so that 1 + e^{-z} stays below 2^126)
__device__ __forceinline__ float sig(float z) { return __fdividef(1.0f, 1.0f + __expf(-fmaxf(z, -80.0f))); }
__device__ __forceinline__ float silu(float z) { return z * sig(z); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = sig(z);
  return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ void stage_params(float *P, const float *__restrict__ params) {
  for (int k = threadIdx.x; k < kNP; k += blockDim.x) P[k < oWo1 ? k : k + kShift] = params[k];
}

__device__ __forceinline__ float dot8(const float *w, const float (&x)[8], float acc) {
  const float4 a = *reinterpret_cast<const float4 *>(w);
  const float4 b = *reinterpret_cast<const float4 *>(w + 4);
  acc = fmaf(a.x, x[0], acc);
  acc = fmaf(a.y, x[1], acc);
  acc = fmaf(a.z, x[2], acc);
  acc = fmaf(a.w, x[3], acc);
  acc = fmaf(b.x, x[4], acc);
  acc = fmaf(b.y, x[5], acc);
  acc = fmaf(b.z, x[6], acc);
  return fmaf(b.w, x[7], acc);
}

__device__ __forceinline__ float dot32(const float *w, const float (&x)[32], float acc) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 a = *reinterpret_cast<const float4 *>(w + 4 * q);
    acc = fmaf(a.x, x[4 * q], acc);
    acc = fmaf(a.y, x[4 * q + 1], acc);
    acc = fmaf(a.z, x[4 * q + 2], acc);
    acc = fmaf(a.w, x[4 * q + 3], acc);
  }
  return acc;
}

// t_ij from the inputs of one bond (weights P in shared memory)
__device__ float hop_forward(const float *P, const float (&C)[8], const float (&u)[8], float nz2) {
  float h1[32];
#pragma unroll
  for (int o = 0; o < 32; ++o) h1[o] = silu(dot8(P + oWe1 + o * 8, u, P[obe1 + o]));
  float e[8];
#pragma unroll
  for (int o = 0; o < 8; ++o) e[o] = C[o] * dot32(P + oWe2 + o * 32, h1, P[obe2 + o]);
  float h2[32];
#pragma unroll
  for (int o = 0; o < 32; ++o) h2[o] = silu(dot8(P + oWh1 + o * 8, e, P[obh1 + o]));
  float y0 = P[obh3], y1 = P[obh3 + 1];
#pragma unroll 4
  for (int o = 0; o < 32; ++o) {
    const float h3 = silu(dot32(P + oWh2 + o * 32, h2, P[obh2 + o]));
    y0 = fmaf(P[oWh3 + o], h3, y0);
    y1 = fmaf(P[oWh3 + 32 + o], h3, y1);
  }
  return y0 * nz2 + y1 * (1.0f - nz2);
}

// MLP_alpha(v_i)[Z_i]
__device__ float onsite_forward(const float *P, const float (&v)[8], int z) {
  float out = P[sbo2 + z];
#pragma unroll 4
  for (int o = 0; o < 32; ++o) out = fmaf(P[sWo2 + z * 32 + o], silu(dot8(P + sWo1 + o * 8, v, P[sbo1 + o])), out);
  return out;
}

__device__ __forceinline__ void load8(const float *__restrict__ p, float (&x)[8]) {
  const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
  const float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
  x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
  x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}

// inputs of bond (i, j): C(r_ij) (species-pair mixing), u = v_i + v_j,
// n_z^2 = (d_z / r)^2 and the bond vector d = r_j + T - r_i (FP32)
__device__ __forceinline__ void bond_inputs(const double *__restrict__ pos, const int32_t *__restrict__ species,
                                            const Box &B, float rcut, const float *sc,
                                            const float *__restrict__ v, int64_t i, int32_t j, float (&C)[8],
                                            float (&u)[8], float &nz2, float3 &d) {
  const int zi = min(max(species[i], 0), 2), zj = min(max(species[j], 0), 2);
  d = bond_vector_f32(B, pos, i, j);
  const float r2 = bond_r2_f32(d);
  bond_descriptor(sqrtf(r2), rcut, sc + (zi * 3 + zj) * 64, C);
  float vi[8], vj[8];
  load8(v + i * 8, vi);
  load8(v + (int64_t)j * 8, vj);
#pragma unroll
  for (int k = 0; k < 8; ++k) u[k] = vi[k] + vj[k];
  nz2 = r2 > 0.0f ? d.z * d.z / r2 : 0.0f;
}

__global__ void env_inputs_kernel(const double *__restrict__ pos, const int32_t *__restrict__ species, int64_t n,
                                  Box B, float rcut, const int64_t *__restrict__ slice_ptr,
                                  const int32_t *__restrict__ col, const int32_t *__restrict__ cnt,
                                  const float *__restrict__ cmix, const float *__restrict__ v,
                                  float *__restrict__ feat) {
  __shared__ float sc[9 * 64];
  load_mixing(sc, cmix);
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t e0 = slice_ptr[i >> 5] + (i & 31);
  const int m = cnt[i];
  for (int s = 0; s < m; ++s) {
    const int64_t e = e0 + 32 * s;
    float C[8], u[8], nz2;
    float3 d;
    bond_inputs(pos, species, B, rcut, sc, v, i, col[e], C, u, nz2, d);
    float *f = feat + e * kNF;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      f[k] = C[k];
      f[8 + k] = u[k];
    }
    f[16] = nz2;
    f[17] = d.x;
    f[18] = d.y;
    f[19] = d.z;
  }
}

// H from stored inputs (training) or from positions (inference), one thread
// per row; padding slots are left untouched
template <typename valT, bool FROM_POS>
__global__ void __launch_bounds__(128) env_forward_kernel(
    int64_t n, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ cnt,
    const float *__restrict__ feat, const double *__restrict__ pos, const int32_t *__restrict__ species, Box B,
    float rcut, const int32_t *__restrict__ col, const float *__restrict__ cmix, const float *__restrict__ v,
    const float *__restrict__ params, const float *__restrict__ eps0, valT *__restrict__ val,
    valT *__restrict__ diag) {
  __shared__ __align__(16) float P[kNPs];
  __shared__ float sc[9 * 64];
  stage_params(P, params);
  if (FROM_POS) load_mixing(sc, cmix);
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e0 = slice_ptr[i >> 5] + (i & 31);
    const int m = cnt[i];
    for (int s = 0; s < m; ++s) {
      const int64_t e = e0 + 32 * s;
      float C[8], u[8], nz2;
      if (FROM_POS) {
        float3 d;
        bond_inputs(pos, species, B, rcut, sc, v, i, col[e], C, u, nz2, d);
      } else {
        load8(feat + e * kNF, C);
        load8(feat + e * kNF + 8, u);
        nz2 = feat[e * kNF + 16];
      }
      val[e] = (valT)hop_forward(P, C, u, nz2);
    }
    if (diag) {
      float vi[8];
      load8(v + i * 8, vi);
      const int z = min(max(species[i], 0), 2);
      diag[i] = (valT)(eps0[z] + onsite_forward(P, vi, z));
    }
  }
}

// ------------------------------------------------------------------ tensor cores
//
// The hopping network of inference (H straight from positions) on the
// 5th-generation tensor cores: BF16 operands, FP32 accumulation in TMEM.  A
// CTA of 4 warps owns tiles of 128 SELL slots (4 slot columns of 32 rows =
// the 128 TMEM lanes); thread t builds the inputs of slot t and owns row t
// of every accumulator.  Per tile (biases of the 8-wide inputs ride on a
// constant-1 column of the K = 16 operand):
//   [u, 1, 0]  (128 x 16) . [We1 | be1]^T           -> D1 (32 columns)
//   h1 = silu(D1)  (128 x 32) . We2^T (8 rows + 8 zero rows) -> D2 (16 columns)
//   e = C (D2[:, :8] + be2);  [e, 1, 0] . [Wh1 | bh1]^T     -> D3 (32 columns)
//   h2 = silu(D3)  (128 x 32) . Wh2^T                 -> D4 (32 columns)
//   h3 = silu(D4 + bh2)  (128 x 32) . Wh3^T (2 rows + 14 zero rows) -> D5 (16 columns)
//   y = D5[:, :2] + bh3;  t = y0 n_z^2 + y1 (1 - n_z^2)  (FP32)
// SiLU here is h + h tanh(h) with h = z/2 (the hardware tanh approximation);
// the weights of the layers followed by SiLU are stored times 1/2, so the
// accumulators hold h directly; h1, h2 and h3 are formed in BF16x2
// arithmetic (they are BF16 operands of the next MMA anyway).
// One thread issues each layer's MMAs and commits them to an mbarrier that
// every thread waits on (bounded; on timeout flags[0] |= 2, the CTA drains
// its MMAs, frees its TMEM and stops).  D3 and D5 reuse D1's columns and D4
// D2's once their loads have completed, so a CTA holds 64 TMEM columns; the
// shared-memory request keeps at most 7 CTAs (448 columns) on an SM.  The
// onsite network (one per row) stays on the FP32 pipes (env_onsite_kernel).
using bf16 = __nv_bfloat16;

struct EnvTcSmem {
  bf16 w1[32 * 16];   // [We1 | be1 | 0]
  bf16 w2[16 * 32];   // We2, rows 8..15 zero
  bf16 w3[32 * 16];   // [Wh1 | bh1 | 0]
  bf16 w4[32 * 32];   // Wh2
  bf16 w5[16 * 32];   // Wh3, rows 2..15 zero
  bf16 a16[128 * 16];  // layer 1 and layer 3 inputs
  bf16 a32[128 * 32];  // layer 2, 4 and 5 inputs
  float be2[8], bh2[32], bh3[2];   // bh2 holds bh2 / 2
  float sc[9 * 64];
  uint64_t bar;
  uint32_t tmem;
};
constexpr int kEnvTcCols = 64;
constexpr int kEnvTcCtasPerSm = 6;   // 6 x 64 of the 512 TMEM columns
constexpr size_t kEnvTcSmemBytes = 30 * 1024;   // >= sizeof + alignment; at most 7 CTAs per SM
static_assert(sizeof(EnvTcSmem) + 128 <= kEnvTcSmemBytes, "env tensor-core shared memory");
constexpr long long kEnvTcPolls = 1ll << 22;


__device__ __forceinline__ uint32_t pack2_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  uint32_t u;
  memcpy(&u, &v, 4);
  return u;
}

// eight values of row r at columns k0 .. k0 + 7 of a K-major core-matrix tile
__device__ __forceinline__ void env_store8(bf16 *tile, int r, int k0, int kdim, const float (&x)[8]) {
  const uint4 u = make_uint4(pack2_bf16(x[0], x[1]), pack2_bf16(x[2], x[3]), pack2_bf16(x[4], x[5]),
                             pack2_bf16(x[6], x[7]));
  *reinterpret_cast<uint4 *>(tile + tc::core_index(r, k0, kdim)) = u;
}

// columns 8..15 of a K = 16 row: the constant 1 (bias) and zeros
__device__ __forceinline__ void env_store_one(bf16 *tile, int r) {
  const uint4 u = make_uint4(pack2_bf16(1.0f, 0.0f), 0u, 0u, 0u);
  *reinterpret_cast<uint4 *>(tile + tc::core_index(r, 8, 16)) = u;
}

__device__ __forceinline__ void env_operands_ready() {
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
}

__device__ __forceinline__ bool env_layer_wait(EnvTcSmem &S, uint32_t &phase, int *flags) {
  const bool ok = __syncthreads_and(tc::mbar_wait(&S.bar, phase, kEnvTcPolls)) != 0;
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(flags, 2);
    tc::mbar_wait(&S.bar, phase, kEnvTcPolls);   // drain the MMAs in flight before TMEM is freed
  }
  phase ^= 1u;
  tc::fence_after_sync();
  return ok;
}

// SiLU of two pre-activations given as h = z/2 (the layer's weights carry
// the factor 1/2, exactly), as a packed BF16 pair: h + h tanh h in BF16x2
// arithmetic (one rounding of h, the hardware tanh, one fused rounding)
__device__ __forceinline__ uint32_t silu2_half_bf16(float h0, float h1) {
  const uint32_t h = pack2_bf16(h0, h1);
  uint32_t t, y;
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(h));
  asm("fma.rn.bf16x2 %0, %1, %2, %1;" : "=r"(y) : "r"(h), "r"(t));
  return y;
}

// the 32 accumulator columns (h = z/2) at taddr of this thread's lane,
// plus a bias (already halved) when BIAS, through SiLU, as row r of the
// K = 32 operand
template <bool BIAS>
__device__ __forceinline__ void env_silu_row32(uint32_t taddr, bf16 *a32, int r, const float *bias) {
#pragma unroll
  for (int c = 0; c < 32; c += 16) {
    float d[16];
    tc::ld16(taddr + (uint32_t)c, d);
    if (BIAS) {
#pragma unroll
      for (int j = 0; j < 16; ++j) d[j] += bias[c + j];
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint4 u = make_uint4(silu2_half_bf16(d[8 * h], d[8 * h + 1]), silu2_half_bf16(d[8 * h + 2], d[8 * h + 3]),
                                 silu2_half_bf16(d[8 * h + 4], d[8 * h + 5]),
                                 silu2_half_bf16(d[8 * h + 6], d[8 * h + 7]));
      *reinterpret_cast<uint4 *>(a32 + tc::core_index(r, c + 8 * h, 32)) = u;
    }
  }
}

// val of every real SELL element from positions (tensor cores; see above)
template <typename valT>
__global__ void __launch_bounds__(128, kEnvTcCtasPerSm) env_hopping_tc_kernel(
    int64_t n, int64_t n_slices, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ cnt,
    const float4 *__restrict__ ph, const float4 *__restrict__ pl, const int32_t *__restrict__ species, BoxPair B,
    float rcut, const int32_t *__restrict__ col, const float *__restrict__ cmix, const float *__restrict__ v,
    const float *__restrict__ params, valT *__restrict__ val, int *__restrict__ flags) {
  extern __shared__ __align__(128) unsigned char env_raw[];
  EnvTcSmem &S = *reinterpret_cast<EnvTcSmem *>(env_raw + ((128 - (tc::smem_addr(env_raw) & 127)) & 127));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // layers followed by SiLU carry the factor 1/2 (exact in BF16): their
  // accumulators hold h = z/2
  for (int q = tid; q < 32 * 16; q += 128) {
    const int o = q >> 4, k = q & 15;
    const float w1 = k < 8 ? params[oWe1 + o * 8 + k] : (k == 8 ? params[obe1 + o] : 0.0f);
    const float w3 = k < 8 ? params[oWh1 + o * 8 + k] : (k == 8 ? params[obh1 + o] : 0.0f);
    S.w1[tc::core_index(o, k, 16)] = __float2bfloat16_rn(0.5f * w1);
    S.w3[tc::core_index(o, k, 16)] = __float2bfloat16_rn(0.5f * w3);
  }
  for (int q = tid; q < 16 * 32; q += 128) {
    const int o = q >> 5, k = q & 31;
    S.w2[tc::core_index(o, k, 32)] = __float2bfloat16_rn(o < 8 ? params[oWe2 + o * 32 + k] : 0.0f);
  }
  for (int q = tid; q < 32 * 32; q += 128)
    S.w4[tc::core_index(q >> 5, q & 31, 32)] = __float2bfloat16_rn(0.5f * params[oWh2 + q]);
  for (int q = tid; q < 16 * 32; q += 128) {
    const int o = q >> 5, k = q & 31;
    S.w5[tc::core_index(o, k, 32)] = __float2bfloat16_rn(o < 2 ? params[oWh3 + o * 32 + k] : 0.0f);
  }
  if (tid < 8) S.be2[tid] = params[obe2 + tid];
  if (tid < 32) S.bh2[tid] = 0.5f * params[obh2 + tid];
  if (tid < 2) S.bh3[tid] = params[obh3 + tid];
  load_mixing(S.sc, cmix);
  env_store_one(S.a16, tid);   // columns 8..15 of this thread's K = 16 row, for every tile
  if (tid == 0) tc::mbar_init(&S.bar, 1);
  if (warp == 0) tc::alloc(&S.tmem, kEnvTcCols);
  env_operands_ready();
  const uint32_t tmem = S.tmem;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's TMEM lanes
  const uint32_t id32 = tc::idesc_bf16(128, 32), id16 = tc::idesc_bf16(128, 16);

  // tiles of 4 slot groups (32 slots of one slice each), contiguous per CTA
  const int64_t slots = slice_ptr[n_slices];
  const int64_t tiles = ((slots >> 5) + 3) >> 2;
  const int64_t t0 = tiles * blockIdx.x / gridDim.x, t1 = tiles * (blockIdx.x + 1) / gridDim.x;
  // this warp's slice: the last slice starting at or before its first slot
  int64_t k = 0;
  {
    const int64_t e0 = (4 * t0 + warp) * 32;
    int64_t hi = n_slices;
    while (hi - k > 1) {
      const int64_t mid = (k + hi) >> 1;
      if (slice_ptr[mid] <= e0) k = mid;
      else hi = mid;
    }
  }
  uint32_t phase = 0;
  bool ok = true;
  for (int64_t t = t0; t < t1 && ok; ++t) {
    const int64_t e0 = (4 * t + warp) * 32;
    while (k + 1 < n_slices && slice_ptr[k + 1] <= e0) ++k;
    const int64_t e = e0 + lane;
    const int64_t i = k * 32 + lane;
    const int slot = static_cast<int>((e0 - slice_ptr[k]) >> 5);
    const bool valid = e0 < slots && i < n && slot < cnt[i];
    float C[8], nz2 = 0.0f;
    {
      float u[8];
      if (valid) {
        const int32_t j = col[e];
        const int zi = min(max(species[i], 0), 2), zj = min(max(species[j], 0), 2);
        const float3 d = bond_vector_pair(B, ph, pl, i, j);
        const float r2 = bond_r2_f32(d);
        bond_descriptor(sqrtf(r2), rcut, S.sc + (zi * 3 + zj) * 64, C);
        float vi[8], vj[8];
        load8(v + i * 8, vi);
        load8(v + (int64_t)j * 8, vj);
#pragma unroll
        for (int k = 0; k < 8; ++k) u[k] = vi[k] + vj[k];
        nz2 = r2 > 0.0f ? d.z * d.z / r2 : 0.0f;
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) C[j] = u[j] = 0.0f;
      }
      env_store8(S.a16, tid, 0, 16, u);
    }
    env_operands_ready();
    if (tid == 0) {
      tc::mma_bf16(tmem, tc::desc_kmajor(S.a16, 16), tc::desc_kmajor(S.w1, 16), id32, false);
      tc::commit(&S.bar);
    }
    if (!(ok = env_layer_wait(S, phase, flags))) break;
    env_silu_row32<false>(tl, S.a32, tid, nullptr);   // h1
    env_operands_ready();
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < 2; ++ks)
        tc::mma_bf16(tmem + 32, tc::desc_kmajor(S.a32 + ks * 128, 32), tc::desc_kmajor(S.w2 + ks * 128, 32), id16,
                     ks > 0);
      tc::commit(&S.bar);
    }
    if (!(ok = env_layer_wait(S, phase, flags))) break;
    {
      float d[16], x[8];
      tc::ld16(tl + 32u, d);
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = C[j] * (d[j] + S.be2[j]);
      env_store8(S.a16, tid, 0, 16, x);   // columns 8..15 still hold [1, 0]
    }
    env_operands_ready();
    if (tid == 0) {
      tc::mma_bf16(tmem, tc::desc_kmajor(S.a16, 16), tc::desc_kmajor(S.w3, 16), id32, false);
      tc::commit(&S.bar);
    }
    if (!(ok = env_layer_wait(S, phase, flags))) break;
    env_silu_row32<false>(tl, S.a32, tid, nullptr);   // h2
    env_operands_ready();
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < 2; ++ks)
        tc::mma_bf16(tmem + 32, tc::desc_kmajor(S.a32 + ks * 128, 32), tc::desc_kmajor(S.w4 + ks * 128, 32), id32,
                     ks > 0);
      tc::commit(&S.bar);
    }
    if (!(ok = env_layer_wait(S, phase, flags))) break;
    env_silu_row32<true>(tl + 32u, S.a32, tid, S.bh2);   // h3
    env_operands_ready();
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < 2; ++ks)
        tc::mma_bf16(tmem, tc::desc_kmajor(S.a32 + ks * 128, 32), tc::desc_kmajor(S.w5 + ks * 128, 32), id16,
                     ks > 0);
      tc::commit(&S.bar);
    }
    if (!(ok = env_layer_wait(S, phase, flags))) break;
    float y[2];
    tc::ld2(tl, y);
    y[0] += S.bh3[0];
    y[1] += S.bh3[1];
    if (valid) val[e] = (valT)(y[0] * nz2 + y[1] * (1.0f - nz2));
    tc::fence_before_sync();   // D5 read before the next tile's layer 1 overwrites it
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, kEnvTcCols);
}

// diag[i] = eps0[Z_i] + MLP_alpha(v_i)[Z_i], one thread per row (FP32)
template <typename valT>
__global__ void __launch_bounds__(128) env_onsite_kernel(int64_t n, const float *__restrict__ v,
                                                         const int32_t *__restrict__ species,
                                                         const float *__restrict__ params,
                                                         const float *__restrict__ eps0, valT *__restrict__ diag) {
  __shared__ __align__(16) float P[kNPs];
  stage_params(P, params);
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float vi[8];
    load8(v + i * 8, vi);
    const int z = min(max(species[i], 0), 2);
    diag[i] = (valT)(eps0[z] + onsite_forward(P, vi, z));
  }
}

// ------------------------------------------------------------------ backward
//
// A CTA of 64 threads takes tiles of 64 items (SELL slots, or rows for the
// onsite network).  Phase 1: each thread runs its item's forward and
// backward pass and leaves, in its shared-memory row, every layer's input
// and output delta (a constant-1 slot serves the biases).  Phase 2: thread t
// owns parameters t, t + 64, ... and adds sum over the tile of delta[o] *
// input[i] into registers.  Rows have an odd stride (no bank conflicts).
constexpr int kBT = 64;
constexpr int kRow = 221;
constexpr int kOwn = (kNP + kBT - 1) / kBT;  // 37
// edge item row: u | dz1 | h1 | dm | e | dz2 | h2 | dz3 | h3 | dy | 1 | 0
constexpr int sU = 0, sDZ1 = 8, sH1 = 40, sDM = 72, sE = 80, sDZ2 = 88, sH2 = 120, sDZ3 = 152, sH3 = 184,
              sDY = 216, sOne = 218, sZero = 219;
// onsite item row: v | dz | h | dout
constexpr int rV = 0, rDZ = 8, rH = 40, rDO = 72;

// shared-memory slots of parameter p for an item kind: input slot and delta
// slot; delta = sZero when the item kind does not touch p
__device__ __forceinline__ void param_slots(int p, bool rows, int &in, int &dl) {
  in = sOne;
  dl = sZero;
  if (!rows) {
    if (p < obe1) { dl = sDZ1 + (p - oWe1) / 8; in = sU + (p - oWe1) % 8; }
    else if (p < oWe2) { dl = sDZ1 + (p - obe1); }
    else if (p < obe2) { dl = sDM + (p - oWe2) / 32; in = sH1 + (p - oWe2) % 32; }
    else if (p < oWh1) { dl = sDM + (p - obe2); }
    else if (p < obh1) { dl = sDZ2 + (p - oWh1) / 8; in = sE + (p - oWh1) % 8; }
    else if (p < oWh2) { dl = sDZ2 + (p - obh1); }
    else if (p < obh2) { dl = sDZ3 + (p - oWh2) / 32; in = sH2 + (p - oWh2) % 32; }
    else if (p < oWh3) { dl = sDZ3 + (p - obh2); }
    else if (p < obh3) { dl = sDY + (p - oWh3) / 32; in = sH3 + (p - oWh3) % 32; }
    else if (p < oWo1) { dl = sDY + (p - obh3); }
  } else {
    if (p < oWo1) return;
    if (p < obo1) { dl = rDZ + (p - oWo1) / 8; in = rV + (p - oWo1) % 8; }
    else if (p < oWo2) { dl = rDZ + (p - obo1); }
    else if (p < obo2) { dl = rDO + (p - oWo2) / 32; in = rH + (p - oWo2) % 32; }
    else { dl = rDO + (p - obo2); }
  }
}

// forward + backward of one bond, activations and deltas into row R
__device__ void hop_backward_item(const float *P, float *R, const float (&C)[8], const float (&u)[8], float nz2,
                                  float g) {
#pragma unroll
  for (int k = 0; k < 8; ++k) R[sU + k] = u[k];
  for (int o = 0; o < 32; ++o) {
    float z = P[obe1 + o];
#pragma unroll
    for (int i = 0; i < 8; ++i) z = fmaf(P[oWe1 + o * 8 + i], u[i], z);
    R[sH1 + o] = silu(z);
    R[sDZ1 + o] = dsilu(z);  // multiplier, becomes dz1 below
  }
  for (int o = 0; o < 8; ++o) {
    float z = P[obe2 + o];
    for (int i = 0; i < 32; ++i) z = fmaf(P[oWe2 + o * 32 + i], R[sH1 + i], z);
    R[sE + o] = C[o] * z;
  }
  for (int o = 0; o < 32; ++o) {
    float z = P[obh1 + o];
#pragma unroll
    for (int i = 0; i < 8; ++i) z = fmaf(P[oWh1 + o * 8 + i], R[sE + i], z);
    R[sH2 + o] = silu(z);
    R[sDZ2 + o] = dsilu(z);
  }
  for (int o = 0; o < 32; ++o) {
    float z = P[obh2 + o];
    for (int i = 0; i < 32; ++i) z = fmaf(P[oWh2 + o * 32 + i], R[sH2 + i], z);
    R[sH3 + o] = silu(z);
    R[sDZ3 + o] = dsilu(z);
  }
  // backward
  const float dy0 = g * nz2, dy1 = g * (1.0f - nz2);
  R[sDY] = dy0;
  R[sDY + 1] = dy1;
  for (int i = 0; i < 32; ++i)
    R[sDZ3 + i] *= fmaf(P[oWh3 + i], dy0, P[oWh3 + 32 + i] * dy1);
  for (int i = 0; i < 32; ++i) {
    float s = 0.0f;
    for (int o = 0; o < 32; ++o) s = fmaf(P[oWh2 + o * 32 + i], R[sDZ3 + o], s);
    R[sDZ2 + i] *= s;
  }
  for (int i = 0; i < 8; ++i) {
    float s = 0.0f;
    for (int o = 0; o < 32; ++o) s = fmaf(P[oWh1 + o * 8 + i], R[sDZ2 + o], s);
    R[sDM + i] = s * C[i];
  }
  for (int i = 0; i < 32; ++i) {
    float s = 0.0f;
#pragma unroll
    for (int o = 0; o < 8; ++o) s = fmaf(P[oWe2 + o * 32 + i], R[sDM + o], s);
    R[sDZ1 + i] *= s;
  }
}

__device__ void onsite_backward_item(const float *P, float *R, const float (&v)[8], int z, float g) {
#pragma unroll
  for (int k = 0; k < 8; ++k) R[rV + k] = v[k];
  for (int o = 0; o < 32; ++o) {
    const float s = dot8(P + sWo1 + o * 8, v, P[sbo1 + o]);
    R[rH + o] = silu(s);
    R[rDZ + o] = dsilu(s) * P[sWo2 + z * 32 + o] * g;
  }
  for (int a = 0; a < 3; ++a) R[rDO + a] = a == z ? g : 0.0f;
}

template <bool ROWS>
__global__ void __launch_bounds__(kBT) env_backward_kernel(
    int64_t n, int64_t n_slices, int64_t total, const int64_t *__restrict__ slice_ptr,
    const int32_t *__restrict__ cnt, const float *__restrict__ feat, const float *__restrict__ v,
    const int32_t *__restrict__ species, const float *__restrict__ params, const float *__restrict__ g_val,
    const float *__restrict__ g_diag, float *__restrict__ partial) {
  extern __shared__ __align__(16) float smem[];
  float *P = smem;
  float *rows = smem + kNPs;
  stage_params(P, params);
  float *R = rows + threadIdx.x * kRow;
  R[sOne] = 1.0f;
  R[sZero] = 0.0f;
  float acc[kOwn];
#pragma unroll
  for (int m = 0; m < kOwn; ++m) acc[m] = 0.0f;
  const int64_t items = ROWS ? n : total;
  const int64_t tiles = (items + kBT - 1) / kBT;
  __syncthreads();
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t it = tile * kBT + threadIdx.x;
    if (ROWS) {
      float vi[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      float g = 0.0f;
      int z = 0;
      if (it < n) {
        g = g_diag[it];
        load8(v + it * 8, vi);
        z = min(max(species[it], 0), 2);
      }
      onsite_backward_item(P, R, vi, z, g);
    } else {
      // locate the slot's slice, row and position in the row
      float C[8] = {0, 0, 0, 0, 0, 0, 0, 0}, u[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      float nz2 = 0.0f, g = 0.0f;
      if (it < total) {
        int64_t lo = 0, hi = n_slices - 1;
        while (lo < hi) {
          const int64_t mid = (lo + hi + 1) >> 1;
          if (slice_ptr[mid] <= it) lo = mid;
          else hi = mid - 1;
        }
        const int64_t off = it - slice_ptr[lo];
        const int64_t row = lo * 32 + (off & 31);
        const int s = (int)(off >> 5);
        if (row < n && s < cnt[row]) {
          load8(feat + it * kNF, C);
          load8(feat + it * kNF + 8, u);
          nz2 = feat[it * kNF + 16];
          g = g_val[it];
        }
      }
      hop_backward_item(P, R, C, u, nz2, g);
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < kOwn; ++m) {
      const int p = threadIdx.x + kBT * m;
      if (p >= kNP) break;
      int in, dl;
      param_slots(p, ROWS, in, dl);
      if (dl == sZero) continue;
      float s = 0.0f;
      for (int k = 0; k < kBT; ++k) s = fmaf(rows[k * kRow + dl], rows[k * kRow + in], s);
      acc[m] += s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < kOwn; ++m) {
    const int p = threadIdx.x + kBT * m;
    if (p < kNP) partial[(int64_t)blockIdx.x * kNP + p] = acc[m];
  }
}

// grad[p] = sum over the partial rows in a fixed order: warp w of a CTA adds
// rows w, w + 8, ... for 32 parameters, then the 8 warp sums in order
__global__ void __launch_bounds__(256) partial_sum_kernel(const float *__restrict__ partial, int nblocks,
                                                          float *__restrict__ grad) {
  __shared__ double part[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int p = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (p < kNP)
    for (int b = w; b < nblocks; b += 8) s += (double)partial[(int64_t)b * kNP + p];
  part[w][lane] = s;
  __syncthreads();
  if (w == 0 && p < kNP) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += part[k][lane];
    grad[p] = (float)t;
  }
}

// ------------------------------------------------------------------ Bloch bands

// butterfly sums: every lane ends with the same two totals, bit for bit
__device__ __forceinline__ void warp_sum2(float &a, float &b) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
}

// The CTA that solves one Bloch matrix (n up to 64).
struct CtaGroup {
  float *red;  // [16] shared scratch for the reductions
  __device__ __forceinline__ int rank() const { return threadIdx.x; }
  __device__ __forceinline__ int size() const { return blockDim.x; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ void sum2(float &a, float &b) const {
    warp_sum2(a, b);
    if ((threadIdx.x & 31) == 0) {
      red[threadIdx.x >> 5] = a;
      red[8 + (threadIdx.x >> 5)] = b;
    }
    __syncthreads();
    a = 0.0f;
    b = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[w];
      b += red[8 + w];
    }
    __syncthreads();
  }
};

// players a < b of pair pp in round `round` of the circle method over m
// players (player 0 fixed, the others rotating)
__device__ __forceinline__ void round_pair(int pp, int round, int m, int &a, int &b) {
  a = pp == 0 ? 0 : 1 + (pp - 1 + round) % (m - 1);
  b = 1 + (m - 2 - pp + round) % (m - 1);
  if (a > b) {
    const int t = a;
    a = b;
    b = t;
  }
}

// H(k) of cell c, cyclic Jacobi, ascending eigenvalues and their vectors
// written out.  Shared memory: A and V [n][n+1], rot and nd [n/2 + 1].
// Returns error bits: 1 = a neighbour outside the cell's rows, 2 = not
// converged in max_sweeps, 4 = a row with more than kMaxCnt neighbours.
template <class G>
__device__ int bloch_solve(const G &g, float2 *A, float2 *V, float4 *rot, float2 *nd, int n, int c, int q,
                           int rows_per_cell, const int64_t *__restrict__ slice_ptr,
                           const int32_t *__restrict__ col, const int32_t *__restrict__ cnt,
                           const float *__restrict__ feat, const float *__restrict__ val,
                           const float *__restrict__ diag, int n_k, const float *__restrict__ kpts, int max_sweeps,
                           float *__restrict__ evals, float2 *__restrict__ evecs) {
  const int ld = n + 1, tid = g.rank(), gs = g.size();
  const float3 k = make_float3(kpts[3 * q], kpts[3 * q + 1], kpts[3 * q + 2]);
  int err = 0;
  for (int idx = tid; idx < n * ld; idx += gs) {
    A[idx] = make_float2(0.0f, 0.0f);
    V[idx] = make_float2(idx / ld == idx % ld ? 1.0f : 0.0f, 0.0f);
  }
  g.sync();
  // Bloch sum: every stored neighbour adds t e^{i k.d}; one thread per row
  for (int i = tid; i < n; i += gs) {
    const int64_t row = (int64_t)c * rows_per_cell + i;
    const int64_t e0 = slice_ptr[row >> 5] + (row & 31);
    const int m = cnt[row];
    if (m > kMaxCnt) err |= 4;
    for (int s = 0; s < m; ++s) {
      const int64_t e = e0 + 32 * s;
      const int64_t j = (int64_t)col[e] - (int64_t)c * rows_per_cell;
      if (j < 0 || j >= n) {
        err |= 1;
        continue;
      }
      const float *f = feat + e * kNF;
      float sn, cs;
      sincosf(k.x * f[17] + k.y * f[18] + k.z * f[19], &sn, &cs);
      const float t = val[e];
      float2 &a = A[i * ld + j];
      a.x = fmaf(t, cs, a.x);
      a.y = fmaf(t, sn, a.y);
    }
    // the diagonal of a Hermitian matrix is real
    A[i * ld + i] = make_float2(A[i * ld + i].x + (diag ? diag[row] : 0.0f), 0.0f);
  }
  g.sync();

  const int m = (n + 1) & ~1;  // players, with one idle slot when n is odd
  const int half = m / 2;
  bool converged = false;
  for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
    for (int round = 0; round < m - 1; ++round) {
      for (int pp = tid; pp < half; pp += gs) {
        int a, b;
        round_pair(pp, round, m, a, b);
        float4 r = make_float4(1.0f, 0.0f, 1.0f, 0.0f);
        float2 dg = make_float2(0.0f, 0.0f);
        if (b < n) {
          const float2 h = A[a * ld + b];
          const float ah = hypotf(h.x, h.y);
          const float app = A[a * ld + a].x, aqq = A[b * ld + b].x;
          dg = make_float2(app, aqq);
          if (ah > 0.0f) {
            const float tau = (aqq - app) / (2.0f * ah);
            const float t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
            // correctly rounded square root and divide: the rotation stays
            // orthogonal to rounding (no drift of the norms over the sweeps)
            const float cth = 1.0f / sqrtf(fmaf(t, t, 1.0f));
            r = make_float4(cth, t * cth, h.x / ah, h.y / ah);
            // rotated diagonal in closed form (Rutishauser)
            dg = make_float2(app - t * ah, aqq + t * ah);
          }
        }
        rot[pp] = r;
        nd[pp] = dg;
      }
      g.sync();
      // rows: A <- U^H A  (new_p = c A_p - s e^{i phi} A_q, new_q = s A_p + c e^{i phi} A_q)
      for (int idx = tid; idx < half * n; idx += gs) {
        const int pp = idx / n, j = idx % n;
        int a, b;
        round_pair(pp, round, m, a, b);
        if (b >= n) continue;
        const float4 r = rot[pp];
        const float2 x = A[a * ld + j], y = A[b * ld + j];
        const float2 ey = make_float2(r.z * y.x - r.w * y.y, r.z * y.y + r.w * y.x);
        A[a * ld + j] = make_float2(r.x * x.x - r.y * ey.x, r.x * x.y - r.y * ey.y);
        A[b * ld + j] = make_float2(r.y * x.x + r.x * ey.x, r.y * x.y + r.x * ey.y);
      }
      g.sync();
      // columns: A <- A U and V <- V U  (new col p = c A_p - s e^{-i phi} A_q,
      // new col q = s A_p + c e^{-i phi} A_q)
      for (int idx = tid; idx < 2 * half * n; idx += gs) {
        const int which = idx / (half * n);
        const int rem = idx % (half * n);
        const int pp = rem / n, i = rem % n;
        int a, b;
        round_pair(pp, round, m, a, b);
        if (b >= n) continue;
        const float4 r = rot[pp];
        float2 *M = which ? V : A;
        const float2 x = M[i * ld + a], y = M[i * ld + b];
        const float2 ey = make_float2(r.z * y.x + r.w * y.y, r.z * y.y - r.w * y.x);
        M[i * ld + a] = make_float2(r.x * x.x - r.y * ey.x, r.x * x.y - r.y * ey.y);
        M[i * ld + b] = make_float2(r.y * x.x + r.x * ey.x, r.y * x.y + r.x * ey.y);
      }
      g.sync();
      // the rotated 2 x 2 block: zero off-diagonal, closed-form diagonal
      for (int pp = tid; pp < half; pp += gs) {
        int a, b;
        round_pair(pp, round, m, a, b);
        if (b < n && rot[pp].y != 0.0f) {
          A[a * ld + b] = make_float2(0.0f, 0.0f);
          A[b * ld + a] = make_float2(0.0f, 0.0f);
          A[a * ld + a] = make_float2(nd[pp].x, 0.0f);
          A[b * ld + b] = make_float2(nd[pp].y, 0.0f);
        }
      }
      g.sync();
    }
    // off-diagonal mass against the total
    float off = 0.0f, tot = 0.0f;
    for (int idx = tid; idx < n * n; idx += gs) {
      const int i = idx / n, j = idx % n;
      const float2 a = A[i * ld + j];
      const float s = a.x * a.x + a.y * a.y;
      tot += s;
      if (i != j) off += s;
    }
    g.sum2(off, tot);
    converged = off <= 1e-13f * tot;
  }
  if (!converged) err |= 2;
  // ascending order: rank of each diagonal entry (ties by index)
  const int64_t base = ((int64_t)c * n_k + q) * n;
  for (int i = tid; i < n; i += gs) {
    const float li = A[i * ld + i].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const float lj = A[j * ld + j].x;
      rank += (lj < li) || (lj == li && j < i);
    }
    evals[base + rank] = li;
    for (int a = 0; a < n; ++a) evecs[(base + a) * n + rank] = V[a * ld + i];
  }
  return err;
}

// one CTA per (k-point, cell), n up to 64
__global__ void __launch_bounds__(256) bloch_eigh_kernel(
    int n, int rows_per_cell, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ col,
    const int32_t *__restrict__ cnt, const float *__restrict__ feat, const float *__restrict__ val,
    const float *__restrict__ diag, int n_k, const float *__restrict__ kpts, int max_sweeps,
    float *__restrict__ evals, float2 *__restrict__ evecs, int *__restrict__ flags) {
  extern __shared__ __align__(16) float2 sh[];
  float2 *A = sh;
  float2 *V = A + n * (n + 1);
  float4 *rot = reinterpret_cast<float4 *>(V + n * (n + 1));
  float2 *nd = reinterpret_cast<float2 *>(rot + kMaxBand / 2);
  float *red = reinterpret_cast<float *>(nd + kMaxBand / 2);
  const int err = bloch_solve(CtaGroup{red}, A, V, rot, nd, n, blockIdx.y, blockIdx.x, rows_per_cell, slice_ptr,
                              col, cnt, feat, val, diag, n_k, kpts, max_sweeps, evals, evecs);
  if (err) atomicOr(flags, err);
}

// One warp per (cell, k-point) for n up to 32: lane j owns column j in the
// row updates and row j in the column updates, so a round is a loop over
// the n/2 pairs with no index arithmetic and only warp-level
// synchronisation; kWarpsEigh matrices per CTA.
constexpr int kWarpsEigh = 4;
__host__ __device__ constexpr size_t eigh_warp_bytes(int n) {
  return ((size_t)2 * n * (n + 1) * sizeof(float2) + 16 * (sizeof(float4) + sizeof(float2) + 2 * sizeof(int)) + 15) /
         16 * 16;
}

__device__ int bloch_solve_warp(float2 *A, float2 *V, float4 *rot, float2 *nd, int *pa, int *pb, int n, int c, int q,
                                int rows_per_cell, const int64_t *__restrict__ slice_ptr,
                                const int32_t *__restrict__ col, const int32_t *__restrict__ cnt,
                                const float *__restrict__ feat, const float *__restrict__ val,
                                const float *__restrict__ diag, int n_k, const float *__restrict__ kpts,
                                int max_sweeps, float *__restrict__ evals, float2 *__restrict__ evecs) {
  const int lane = threadIdx.x & 31, ld = n + 1;
  const float3 k = make_float3(kpts[3 * q], kpts[3 * q + 1], kpts[3 * q + 2]);
  int err = 0;
  if (lane < n) {
    for (int j = 0; j < n; ++j) {
      A[lane * ld + j] = make_float2(0.0f, 0.0f);
      V[lane * ld + j] = make_float2(lane == j ? 1.0f : 0.0f, 0.0f);
    }
    // Bloch sum of row `lane`: every stored neighbour adds t e^{i k.d}
    const int64_t row = (int64_t)c * rows_per_cell + lane;
    const int64_t e0 = slice_ptr[row >> 5] + (row & 31);
    const int m = cnt[row];
    if (m > kMaxCnt) err |= 4;
    for (int s = 0; s < m; ++s) {
      const int64_t e = e0 + 32 * s;
      const int64_t j = (int64_t)col[e] - (int64_t)c * rows_per_cell;
      if (j < 0 || j >= n) {
        err |= 1;
        continue;
      }
      const float *f = feat + e * kNF;
      float sn, cs;
      sincosf(k.x * f[17] + k.y * f[18] + k.z * f[19], &sn, &cs);
      const float t = val[e];
      float2 &a = A[lane * ld + j];
      a.x = fmaf(t, cs, a.x);
      a.y = fmaf(t, sn, a.y);
    }
    A[lane * ld + lane] = make_float2(A[lane * ld + lane].x + (diag ? diag[row] : 0.0f), 0.0f);
  }
  __syncwarp();

  const int m = (n + 1) & ~1;
  const int half = m / 2;
  bool converged = false;
  for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
    for (int round = 0; round < m - 1; ++round) {
      if (lane < half) {
        int a, b;
        round_pair(lane, round, m, a, b);
        float4 r = make_float4(1.0f, 0.0f, 1.0f, 0.0f);
        float2 dg = make_float2(0.0f, 0.0f);
        if (b < n) {
          const float2 h = A[a * ld + b];
          const float ah = hypotf(h.x, h.y);
          const float app = A[a * ld + a].x, aqq = A[b * ld + b].x;
          dg = make_float2(app, aqq);
          if (ah > 0.0f) {
            const float tau = (aqq - app) / (2.0f * ah);
            const float t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
            const float cth = 1.0f / sqrtf(fmaf(t, t, 1.0f));
            r = make_float4(cth, t * cth, h.x / ah, h.y / ah);
            dg = make_float2(app - t * ah, aqq + t * ah);
          }
        } else {
          b = -1;  // idle pair (odd n)
        }
        pa[lane] = a;
        pb[lane] = b;
        rot[lane] = r;
        nd[lane] = dg;
      }
      __syncwarp();
      if (lane < n) {
        // rows a, b at column `lane`: A <- U^H A
        for (int pp = 0; pp < half; ++pp) {
          const int a = pa[pp], b = pb[pp];
          if (b < 0) continue;
          const float4 r = rot[pp];
          const float2 x = A[a * ld + lane], y = A[b * ld + lane];
          const float2 ey = make_float2(r.z * y.x - r.w * y.y, r.z * y.y + r.w * y.x);
          A[a * ld + lane] = make_float2(r.x * x.x - r.y * ey.x, r.x * x.y - r.y * ey.y);
          A[b * ld + lane] = make_float2(r.y * x.x + r.x * ey.x, r.y * x.y + r.x * ey.y);
        }
      }
      __syncwarp();
      if (lane < n) {
        // columns a, b at row `lane`: A <- A U, V <- V U
        for (int pp = 0; pp < half; ++pp) {
          const int a = pa[pp], b = pb[pp];
          if (b < 0) continue;
          const float4 r = rot[pp];
          float2 x = A[lane * ld + a], y = A[lane * ld + b];
          float2 ey = make_float2(r.z * y.x + r.w * y.y, r.z * y.y - r.w * y.x);
          A[lane * ld + a] = make_float2(r.x * x.x - r.y * ey.x, r.x * x.y - r.y * ey.y);
          A[lane * ld + b] = make_float2(r.y * x.x + r.x * ey.x, r.y * x.y + r.x * ey.y);
          x = V[lane * ld + a];
          y = V[lane * ld + b];
          ey = make_float2(r.z * y.x + r.w * y.y, r.z * y.y - r.w * y.x);
          V[lane * ld + a] = make_float2(r.x * x.x - r.y * ey.x, r.x * x.y - r.y * ey.y);
          V[lane * ld + b] = make_float2(r.y * x.x + r.x * ey.x, r.y * x.y + r.x * ey.y);
        }
      }
      __syncwarp();
      if (lane < half) {
        const int a = pa[lane], b = pb[lane];
        if (b >= 0 && rot[lane].y != 0.0f) {
          A[a * ld + b] = make_float2(0.0f, 0.0f);
          A[b * ld + a] = make_float2(0.0f, 0.0f);
          A[a * ld + a] = make_float2(nd[lane].x, 0.0f);
          A[b * ld + b] = make_float2(nd[lane].y, 0.0f);
        }
      }
      __syncwarp();
    }
    float off = 0.0f, tot = 0.0f;
    if (lane < n) {
      for (int j = 0; j < n; ++j) {
        const float2 a = A[lane * ld + j];
        const float s = a.x * a.x + a.y * a.y;
        tot += s;
        if (j != lane) off += s;
      }
    }
    warp_sum2(off, tot);
    converged = off <= 1e-13f * tot;
  }
  if (!converged) err |= 2;
  const int64_t base = ((int64_t)c * n_k + q) * n;
  if (lane < n) {
    const float li = A[lane * ld + lane].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const float lj = A[j * ld + j].x;
      rank += (lj < li) || (lj == li && j < lane);
    }
    evals[base + rank] = li;
    for (int a = 0; a < n; ++a) evecs[(base + a) * n + rank] = V[a * ld + lane];
  }
  return err;
}

__global__ void __launch_bounds__(32 * kWarpsEigh) bloch_eigh_warp_kernel(
    int n, int rows_per_cell, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ col,
    const int32_t *__restrict__ cnt, const float *__restrict__ feat, const float *__restrict__ val,
    const float *__restrict__ diag, int n_cells, int n_k, const float *__restrict__ kpts, int max_sweeps,
    float *__restrict__ evals, float2 *__restrict__ evecs, int *__restrict__ flags) {
  extern __shared__ __align__(16) unsigned char shb[];
  const int w = threadIdx.x >> 5;
  const int64_t mi = (int64_t)blockIdx.x * kWarpsEigh + w;
  if (mi >= (int64_t)n_cells * n_k) return;  // whole warp: no block barrier follows
  unsigned char *base = shb + (size_t)w * eigh_warp_bytes(n);
  float2 *A = reinterpret_cast<float2 *>(base);
  float2 *V = A + n * (n + 1);
  float4 *rot = reinterpret_cast<float4 *>(base + (size_t)2 * n * (n + 1) * sizeof(float2));
  float2 *nd = reinterpret_cast<float2 *>(rot + 16);
  int *pa = reinterpret_cast<int *>(nd + 16);
  int *pb = pa + 16;
  const int c = (int)(mi / n_k), q = (int)(mi % n_k);
  const int err = bloch_solve_warp(A, V, rot, nd, pa, pb, n, c, q, rows_per_cell, slice_ptr, col, cnt, feat, val,
                                   diag, n_k, kpts, max_sweeps, evals, evecs);
  if (err) atomicOr(flags, err);
}

// Eq. 3 over all (cell, k, band) items: stats = {S, sum w D^2, L}; the
// terms in FP32, their sums in FP64
__global__ void __launch_bounds__(1024) band_loss_kernel(int items, int nb, const float *__restrict__ E,
                                                         const float *__restrict__ Eref,
                                                         const float *__restrict__ w, float *__restrict__ dLdE,
                                                         double *__restrict__ stats) {
  __shared__ double red[2][32];
  __shared__ float S_all;
  double s1 = 0.0, s2 = 0.0;
  for (int x = threadIdx.x; x < items; x += blockDim.x) {
    const float d = E[x] - Eref[x];
    const float wb = w[x % nb];
    s1 += (double)(wb * fabsf(d));
    s2 += (double)(wb * d * d);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s1;
    red[1][threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += red[0][k];
      b += red[1][k];
    }
    S_all = (float)a;
    stats[0] = a;
    stats[1] = b;
    stats[2] = a * a + b;
  }
  __syncthreads();
  const float S2 = 2.0f * S_all;
  for (int x = threadIdx.x; x < items; x += blockDim.x) {
    const float d = E[x] - Eref[x];
    const float wb = w[x % nb];
    const float sg = d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f);
    dLdE[x] = wb * fmaf(S2, sg, 2.0f * d);
  }
}

// Hellmann-Feynman: dL/dt_e = sum_k sum_b g_b Re(conj(psi_b[i]) psi_b[j] e^{i k.d_e}),
// dL/deps_i = sum_k sum_b g_b |psi_b[i]|^2; one CTA per cell, k-points in turn
constexpr int kGradItems = kMaxBand * kMaxCnt / 256;  // slots per thread
__global__ void __launch_bounds__(256) band_gradient_kernel(
    int n, int rows_per_cell, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ col,
    const int32_t *__restrict__ cnt, const float *__restrict__ feat, int n_k, const float *__restrict__ kpts,
    const float2 *__restrict__ evecs, const float *__restrict__ dLdE, float *__restrict__ g_val,
    float *__restrict__ g_diag) {
  extern __shared__ float2 sh[];
  const int ld = n + 1;
  float2 *Psi = sh;
  float *g = reinterpret_cast<float *>(Psi + n * ld);
  const int c = blockIdx.x;
  float acc[kGradItems];
#pragma unroll
  for (int m = 0; m < kGradItems; ++m) acc[m] = 0.0f;
  float acc_eps = 0.0f;
  for (int q = 0; q < n_k; ++q) {
    const int64_t base = ((int64_t)c * n_k + q) * n;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) Psi[(idx / n) * ld + idx % n] = evecs[base * n + idx];
    for (int b = threadIdx.x; b < n; b += blockDim.x) g[b] = dLdE[base + b];
    __syncthreads();
    const float kx = kpts[3 * q], ky = kpts[3 * q + 1], kz = kpts[3 * q + 2];
#pragma unroll
    for (int m = 0; m < kGradItems; ++m) {
      const int item = threadIdx.x + 256 * m;
      const int i = item / kMaxCnt, s = item % kMaxCnt;
      if (i >= n) continue;
      const int64_t row = (int64_t)c * rows_per_cell + i;
      if (s >= cnt[row]) continue;
      const int64_t e = slice_ptr[row >> 5] + (row & 31) + 32 * s;
      const int64_t j = (int64_t)col[e] - (int64_t)c * rows_per_cell;
      if (j < 0 || j >= n) continue;
      float zr = 0.0f, zi = 0.0f;
      for (int b = 0; b < n; ++b) {
        const float2 pi = Psi[i * ld + b], pj = Psi[j * ld + b];
        // conj(pi) pj
        zr = fmaf(g[b], pi.x * pj.x + pi.y * pj.y, zr);
        zi = fmaf(g[b], pi.x * pj.y - pi.y * pj.x, zi);
      }
      const float *f = feat + e * kNF;
      float sn, cs;
      sincosf(kx * f[17] + ky * f[18] + kz * f[19], &sn, &cs);
      acc[m] += zr * cs - zi * sn;
    }
    if (threadIdx.x < n) {
      const int i = threadIdx.x;
      float s = 0.0f;
      for (int b = 0; b < n; ++b) {
        const float2 p = Psi[i * ld + b];
        s = fmaf(g[b], p.x * p.x + p.y * p.y, s);
      }
      acc_eps += s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < kGradItems; ++m) {
    const int item = threadIdx.x + 256 * m;
    const int i = item / kMaxCnt, s = item % kMaxCnt;
    if (i >= n) continue;
    const int64_t row = (int64_t)c * rows_per_cell + i;
    if (s >= cnt[row]) continue;
    g_val[slice_ptr[row >> 5] + (row & 31) + 32 * s] = acc[m];
  }
  for (int i = threadIdx.x; i < rows_per_cell; i += blockDim.x)
    g_diag[(int64_t)c * rows_per_cell + i] = i < n ? acc_eps : 0.0f;
}

__global__ void adamw_flat_kernel(int64_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                                  float *__restrict__ v, float lr, float b1, float b2, float eps, float wd, float c1,
                                  float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
  const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] * (1.0f - lr * wd);
  p[i] = pi - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

size_t eigh_smem(int n) {
  return (size_t)2 * n * (n + 1) * sizeof(float2) + kMaxBand / 2 * (sizeof(float4) + sizeof(float2)) + 16 * 4;
}
size_t grad_smem(int n) { return (size_t)n * (n + 1) * sizeof(float2) + n * sizeof(float); }
int backward_grid(int64_t items) {
  const int64_t tiles = (items + kBT - 1) / kBT;
  const int64_t g = (int64_t)sm_count() * 3;
  return (int)(tiles < g ? (tiles > 0 ? tiles : 1) : g);
}
constexpr size_t kBackSmem = (size_t)(kNPs + kBT * kRow) * sizeof(float);

tb_status check_sell(int64_t n, const int64_t *slice_ptr, const int32_t *cnt) {
  TB_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "bad row count");
  TB_REQUIRE(slice_ptr && cnt, "slice_ptr and cnt are required");
  return TB_OK;
}

}  // namespace
}  // namespace gputb

using namespace gputb;

extern "C" tb_status tb_env_edge_inputs(const double *positions, const int32_t *species, int64_t n,
                                        const double *box, const int32_t *pbc, double rcut,
                                        const int64_t *slice_ptr, const int32_t *col, const int32_t *cnt,
                                        const float *cmix, const float *v, float *feat, void *stream) {
  tb_status s = check_sell(n, slice_ptr, cnt);
  if (s != TB_OK) return s;
  TB_REQUIRE(positions && species && cmix && v && feat, "tb_env_edge_inputs: null pointer");
  Box B;
  s = make_box(box, pbc, rcut, &B);
  if (s != TB_OK) return s;
  env_inputs_kernel<<<(unsigned)((n + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
      positions, species, n, B, (float)rcut, slice_ptr, col, cnt, cmix, v, feat);
  TB_CHECK_LAUNCH();
  return TB_OK;
}

namespace {
template <typename valT, bool FROM_POS>
tb_status launch_env_forward(int64_t n, const int64_t *slice_ptr, const int32_t *cnt, const float *feat,
                             const double *pos, const int32_t *species, const Box &B, float rcut,
                             const int32_t *col, const float *cmix, const float *v, const float *params,
                             const float *eps0, void *val, void *diag, cudaStream_t st) {
  // one wave: the resident CTAs of every SM, each striding over the rows
  int occ = 0;
  TB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, env_forward_kernel<valT, FROM_POS>, 128, 0));
  const int64_t want = (n + 127) / 128;
  const int64_t cap = (int64_t)sm_count() * (occ > 0 ? occ : 1);
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  env_forward_kernel<valT, FROM_POS><<<grid, 128, 0, st>>>(n, slice_ptr, cnt, feat, pos, species, B, rcut, col,
                                                          cmix, v, params, eps0, static_cast<valT *>(val),
                                                          static_cast<valT *>(diag));
  TB_CHECK_LAUNCH();
  return TB_OK;
}
}  // namespace

extern "C" tb_status tb_env_forward(int64_t n, const int64_t *slice_ptr, const int32_t *cnt, const float *feat,
                                    const float *v, const int32_t *species, const float *params, const float *eps0,
                                    int32_t precision, void *val, void *diag, void *stream) {
  tb_status s = check_sell(n, slice_ptr, cnt);
  if (s != TB_OK) return s;
  TB_REQUIRE(feat && params && val, "tb_env_forward: null pointer");
  TB_REQUIRE(!diag || (v && species && eps0), "tb_env_forward: diag needs v, species and eps0");
  TB_REQUIRE(precision == TB_F32 || precision == TB_F64, "tb_env_forward: bad precision");
  Box B{};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (precision == TB_F32)
    return launch_env_forward<float, false>(n, slice_ptr, cnt, feat, nullptr, species, B, 0.0f, nullptr, nullptr, v,
                                            params, eps0, val, diag, st);
  return launch_env_forward<double, false>(n, slice_ptr, cnt, feat, nullptr, species, B, 0.0f, nullptr, nullptr, v,
                                           params, eps0, val, diag, st);
}

namespace {
// kernel of tb_build_hamiltonian_env: 0 = tensor cores (default), 1 = FP32 pipes
int g_env_variant = 0;

template <typename valT>
tb_status launch_env_tc(int64_t n, const int64_t *slice_ptr, const int32_t *cnt, const double *pos,
                        const int32_t *species, const Box &B, float rcut, const int32_t *col, const float *cmix,
                        const float *v, const float *params, const float *eps0, void *val, void *diag, int *flags,
                        float4 *ph, float4 *pl, cudaStream_t st) {
  const int64_t n_slices = (n + 31) / 32;
  pos_pair_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pos, n, ph, pl);
  TB_CHECK_LAUNCH();
  // the whole unified L1/shared array as shared memory: room for 7 CTAs of 30 KB
  TB_CUDA(cudaFuncSetAttribute(env_hopping_tc_kernel<valT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kEnvTcSmemBytes));
  TB_CUDA(cudaFuncSetAttribute(env_hopping_tc_kernel<valT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared));
  // persistent: 6 CTAs per SM (the register budget of the launch bounds; the
  // occupancy query reports 1 for this kernel), each taking a contiguous
  // range of 128-slot tiles (empty for the CTAs beyond the tile count)
  const unsigned grid = (unsigned)(sm_count() * kEnvTcCtasPerSm);
  env_hopping_tc_kernel<valT><<<grid, 128, kEnvTcSmemBytes, st>>>(n, n_slices, slice_ptr, cnt, ph, pl, species,
                                                                   box_pair(B), rcut, col, cmix, v, params,
                                                                   static_cast<valT *>(val), flags);
  TB_CHECK_LAUNCH();
  if (diag) {
    const int64_t want = (n + 127) / 128, cap = (int64_t)sm_count() * 8;
    env_onsite_kernel<valT><<<(unsigned)(want < cap ? want : cap), 128, 0, st>>>(n, v, species, params, eps0,
                                                                                static_cast<valT *>(diag));
    TB_CHECK_LAUNCH();
  }
  return TB_OK;
}
}  // namespace

extern "C" size_t tb_build_hamiltonian_env_workspace_size(int64_t n) {
  if (n < 0) return 0;
  return 256 + (size_t)n * 2 * sizeof(float4);   // status word, then the FP32-pair positions
}

extern "C" tb_status tb_build_hamiltonian_env(const double *positions, const int32_t *species, int64_t n,
                                              const double *box, const int32_t *pbc, double rcut,
                                              const int64_t *slice_ptr, const int32_t *col, const int32_t *cnt,
                                              const float *cmix, const float *v, const float *params,
                                              const float *eps0, int32_t precision, void *val, void *diag,
                                              void *workspace, size_t workspace_bytes, void *stream) {
  tb_status s = check_sell(n, slice_ptr, cnt);
  if (s != TB_OK) return s;
  TB_REQUIRE(positions && species && cmix && v && params && eps0 && val,
             "tb_build_hamiltonian_env: null pointer");
  TB_REQUIRE(precision == TB_F32 || precision == TB_F64, "tb_build_hamiltonian_env: bad precision");
  TB_REQUIRE(workspace && (reinterpret_cast<uintptr_t>(workspace) & 255) == 0,
             "tb_build_hamiltonian_env: workspace must be 256-byte aligned");
  if (workspace_bytes < tb_build_hamiltonian_env_workspace_size(n))
    return fail(TB_ERR_WORKSPACE, "tb_build_hamiltonian_env: workspace too small (%zu < %zu)", workspace_bytes,
                tb_build_hamiltonian_env_workspace_size(n));
  Box B;
  s = make_box(box, pbc, rcut, &B);
  if (s != TB_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (g_env_variant == 1) {
    if (precision == TB_F32)
      return launch_env_forward<float, true>(n, slice_ptr, cnt, nullptr, positions, species, B, (float)rcut, col,
                                             cmix, v, params, eps0, val, diag, st);
    return launch_env_forward<double, true>(n, slice_ptr, cnt, nullptr, positions, species, B, (float)rcut, col,
                                            cmix, v, params, eps0, val, diag, st);
  }
  if (n == 0) return TB_OK;
  int *flags = static_cast<int *>(workspace);
  float4 *ph = reinterpret_cast<float4 *>(static_cast<unsigned char *>(workspace) + 256);
  float4 *pl = ph + n;
  TB_CUDA(cudaMemsetAsync(flags, 0, sizeof(int), st));
  s = precision == TB_F32 ? launch_env_tc<float>(n, slice_ptr, cnt, positions, species, B, (float)rcut, col, cmix, v,
                                                 params, eps0, val, diag, flags, ph, pl, st)
                          : launch_env_tc<double>(n, slice_ptr, cnt, positions, species, B, (float)rcut, col, cmix,
                                                  v, params, eps0, val, diag, flags, ph, pl, st);
  if (s != TB_OK) return s;
  int h = 0;
  TB_CUDA(cudaMemcpyAsync(&h, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  TB_CUDA(cudaStreamSynchronize(st));
  if (h & 2) return fail(TB_ERR_TIMEOUT, "tb_build_hamiltonian_env: a tensor-core completion wait timed out");
  return TB_OK;
}

extern "C" tb_status tb_env_set_variant(int32_t variant) {
  TB_REQUIRE(variant == 0 || variant == 1, "tb_env_set_variant: variant must be 0 (tcgen05) or 1 (FP32 pipes)");
  g_env_variant = variant;
  return TB_OK;
}

extern "C" size_t tb_env_backward_workspace_size(int64_t n, int64_t total_elements) {
  if (n < 0 || total_elements < 0) return 0;
  return (size_t)(backward_grid(total_elements) + backward_grid(n)) * kNP * sizeof(float) + 256;
}

extern "C" tb_status tb_env_backward(int64_t n, const int64_t *slice_ptr, const int32_t *cnt, int64_t total_elements,
                                     const float *feat, const float *v, const int32_t *species, const float *params,
                                     const float *g_val, const float *g_diag, float *grad, void *workspace,
                                     size_t workspace_bytes, void *stream) {
  tb_status s = check_sell(n, slice_ptr, cnt);
  if (s != TB_OK) return s;
  TB_REQUIRE(total_elements >= 0 && feat && v && species && params && g_val && g_diag && grad && workspace,
             "tb_env_backward: bad argument");
  if (workspace_bytes < tb_env_backward_workspace_size(n, total_elements))
    return fail(TB_ERR_WORKSPACE, "tb_env_backward: workspace too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int ge = backward_grid(total_elements), gr = backward_grid(n);
  float *partial = static_cast<float *>(workspace);
  const int64_t n_slices = (n + 31) / 32;
  TB_CUDA(cudaFuncSetAttribute(env_backward_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kBackSmem));
  TB_CUDA(cudaFuncSetAttribute(env_backward_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kBackSmem));
  env_backward_kernel<false><<<ge, kBT, kBackSmem, st>>>(n, n_slices, total_elements, slice_ptr, cnt, feat, v,
                                                         species, params, g_val, g_diag, partial);
  TB_CHECK_LAUNCH();
  env_backward_kernel<true><<<gr, kBT, kBackSmem, st>>>(n, n_slices, total_elements, slice_ptr, cnt, feat, v,
                                                        species, params, g_val, g_diag,
                                                        partial + (int64_t)ge * kNP);
  TB_CHECK_LAUNCH();
  partial_sum_kernel<<<(kNP + 31) / 32, 256, 0, st>>>(partial, ge + gr, grad);
  TB_CHECK_LAUNCH();
  return TB_OK;
}

extern "C" tb_status tb_bloch_bands(int32_t n_cells, int32_t n_atoms, int32_t rows_per_cell,
                                    const int64_t *slice_ptr, const int32_t *col, const int32_t *cnt,
                                    const float *feat, const float *val, const float *diag, int32_t n_k,
                                    const float *kpts, int32_t max_sweeps, float *evals, void *evecs,
                                    int32_t *flags, void *stream) {
  TB_REQUIRE(n_cells >= 1 && n_k >= 1 && n_k <= 65535 && n_cells <= 65535, "tb_bloch_bands: bad batch size");
  TB_REQUIRE(n_atoms >= 1 && n_atoms <= kMaxBand, "tb_bloch_bands: n_atoms must be 1..64");
  TB_REQUIRE(rows_per_cell >= n_atoms && rows_per_cell % 32 == 0, "tb_bloch_bands: rows_per_cell must be a multiple of 32 >= n_atoms");
  TB_REQUIRE(max_sweeps >= 1 && max_sweeps <= 100, "tb_bloch_bands: max_sweeps must be 1..100");
  TB_REQUIRE(slice_ptr && col && cnt && feat && val && kpts && evals && evecs && flags,
             "tb_bloch_bands: null pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TB_CUDA(cudaMemsetAsync(flags, 0, sizeof(int32_t), st));
  if (n_atoms <= 32) {
    const size_t smem = kWarpsEigh * eigh_warp_bytes(n_atoms);
    TB_CUDA(cudaFuncSetAttribute(bloch_eigh_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t mats = (int64_t)n_cells * n_k;
    bloch_eigh_warp_kernel<<<(unsigned)((mats + kWarpsEigh - 1) / kWarpsEigh), 32 * kWarpsEigh, smem, st>>>(
        n_atoms, rows_per_cell, slice_ptr, col, cnt, feat, val, diag, n_cells, n_k, kpts, max_sweeps, evals,
        static_cast<float2 *>(evecs), flags);
  } else {
    const size_t smem = eigh_smem(n_atoms);
    TB_CUDA(cudaFuncSetAttribute(bloch_eigh_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    bloch_eigh_kernel<<<dim3(n_k, n_cells), 256, smem, st>>>(n_atoms, rows_per_cell, slice_ptr, col, cnt, feat,
                                                            val, diag, n_k, kpts, max_sweeps, evals,
                                                            static_cast<float2 *>(evecs), flags);
  }
  TB_CHECK_LAUNCH();
  int32_t h = 0;
  TB_CUDA(cudaMemcpyAsync(&h, flags, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  TB_CUDA(cudaStreamSynchronize(st));
  if (h & 1) return fail(TB_ERR_INVALID_ARG, "tb_bloch_bands: a neighbour lies outside its cell's rows");
  if (h & 4) return fail(TB_ERR_ELL_OVERFLOW, "tb_bloch_bands: a row has more than 32 neighbours");
  if (h & 2) return fail(TB_ERR_NOT_CONVERGED, "tb_bloch_bands: Jacobi rotations did not converge in max_sweeps");
  return TB_OK;
}

extern "C" tb_status tb_band_loss(int64_t n_spectra, int32_t n_bands, const float *evals, const float *e_ref,
                                  const float *weights, float *dLdE, double *stats, void *stream) {
  TB_REQUIRE(n_spectra >= 1 && n_bands >= 1 && evals && e_ref && weights && dLdE && stats,
             "tb_band_loss: bad argument");
  TB_REQUIRE(n_spectra * (int64_t)n_bands < (int64_t(1) << 31), "tb_band_loss: more than 2^31 - 1 band energies");
  band_loss_kernel<<<1, 1024, 0, static_cast<cudaStream_t>(stream)>>>((int)(n_spectra * n_bands), n_bands, evals,
                                                                     e_ref, weights, dLdE, stats);
  TB_CHECK_LAUNCH();
  return TB_OK;
}

extern "C" tb_status tb_band_gradient(int32_t n_cells, int32_t n_atoms, int32_t rows_per_cell,
                                      const int64_t *slice_ptr, const int32_t *col, const int32_t *cnt,
                                      const float *feat, int32_t n_k, const float *kpts, const void *evecs,
                                      const float *dLdE, float *g_val, float *g_diag, void *stream) {
  TB_REQUIRE(n_cells >= 1 && n_k >= 1, "tb_band_gradient: bad batch size");
  TB_REQUIRE(n_atoms >= 1 && n_atoms <= kMaxBand, "tb_band_gradient: n_atoms must be 1..64");
  TB_REQUIRE(rows_per_cell >= n_atoms && rows_per_cell % 32 == 0, "tb_band_gradient: bad rows_per_cell");
  TB_REQUIRE(slice_ptr && col && cnt && feat && kpts && evecs && dLdE && g_val && g_diag,
             "tb_band_gradient: null pointer");
  const size_t smem = grad_smem(n_atoms);
  TB_CUDA(cudaFuncSetAttribute(band_gradient_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  band_gradient_kernel<<<n_cells, 256, smem, static_cast<cudaStream_t>(stream)>>>(
      n_atoms, rows_per_cell, slice_ptr, col, cnt, feat, n_k, kpts, static_cast<const float2 *>(evecs), dLdE, g_val,
      g_diag);
  TB_CHECK_LAUNCH();
  return TB_OK;
}

extern "C" tb_status tb_adamw_flat(int64_t n, float *params, const float *grad, float *m, float *v, int64_t step,
                                   double lr, double beta1, double beta2, double eps, double weight_decay,
                                   void *stream) {
  TB_REQUIRE(n >= 1 && params && grad && m && v && step >= 1, "tb_adamw_flat: bad argument");
  const double c1 = 1.0 - std::pow(beta1, (double)step), c2 = 1.0 - std::pow(beta2, (double)step);
  adamw_flat_kernel<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, params, grad, m, v, (float)lr, (float)beta1, (float)beta2, (float)eps, (float)weight_decay, (float)c1,
      (float)c2);
  TB_CHECK_LAUNCH();
  return TB_OK;
}
