// Teacher Hamiltonian in SELL-32 form: the analytic, environment-dependent
// orthogonal pz model (form of Eq. 1, arXiv 2509.06525 Sec. 3) that labels
// the training snapshots and serves as the plain method:
//   t_ij  = P[Z_i,Z_j] exp(-beta (r_ij/a_cc - 1)) (1 + gamma (n_i+n_j-6)/6) f_c(r_ij)
//   f_c(r) = (1 + cos(pi r / r_cut)) / 2 for r < r_cut, else 0
//   eps_i = onsite[Z_i]
// One thread per row walks the row's slots (coalesced across the 32 rows of
// a slice), recomputes the bond length and writes the value in FP32 or FP64:
// for FP64 values from the FP64 minimum image, for FP32 values from the
// positions split into FP32 pairs (r^2 to about 44 bits); the exponential
// and cosine are evaluated in the output precision.
#include <cmath>

#include "geometry.cuh"

namespace gputb {
namespace {

struct TeacherConst {
  double pref[9];
  double onsite[3];
  double a_cc, beta, gamma, rcut, inv_a;
  float2 rc2, a2;   // rcut^2 and a_cc^2 as FP32 pairs
  int n_species;
};

// x - c for pairs, rounded to FP32 (TwoSum of the high parts: no
// cancellation when x is close to c)
__device__ __forceinline__ float pair_diff(float2 x, float2 c) {
  const float2 t = two_sum_f(x.x, -c.x);
  return t.x + (t.y + (x.y - c.y));
}

template <typename valT>
__global__ void teacher_kernel(const double *__restrict__ pos, const float4 *__restrict__ ph,
                               const float4 *__restrict__ pl, const int32_t *__restrict__ species, int64_t n,
                               Box B, BoxPair BP, TeacherConst T, const int64_t *__restrict__ slice_ptr,
                               const int32_t *__restrict__ col, const int32_t *__restrict__ cnt,
                               const int32_t *__restrict__ ncount, valT *__restrict__ val, valT *__restrict__ diag,
                               int *__restrict__ flags) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ((n + 31) >> 5) << 5) return;
  const int64_t sb = slice_ptr[i >> 5];
  const int w = static_cast<int>((slice_ptr[(i >> 5) + 1] - sb) >> 5);
  if (i >= n) {  // phantom rows of the last slice hold value 0
    for (int s = 0; s < w; ++s) val[sb + (i & 31) + 32 * s] = valT(0);
    return;
  }
  const int zi = species[i];
  if (zi < 0 || zi >= T.n_species) atomicOr(flags, 1);
  const int zic = min(max(zi, 0), T.n_species - 1);
  const int ni = ncount[i];
  const int m = cnt[i];
  int64_t e = sb + (i & 31);
  for (int s = 0; s < w; ++s, e += 32) {
    double t = 0.0;
    if (s < m) {
      const int32_t j = col[e];
      const int zj = min(max(species[j], 0), T.n_species - 1);
      if (sizeof(valT) == 8) {
        const double r2 = bond_r2(B, pos, i, j);
        const double r = sqrt(r2);
        const double env = 1.0 + T.gamma * ((double)(ni + ncount[j]) - 6.0) / 6.0;
        const double fc = r < T.rcut ? 0.5 * (1.0 + cos(M_PI * r / T.rcut)) : 0.0;
        t = T.pref[zic * 3 + zj] * exp(-T.beta * (r / T.a_cc - 1.0)) * env * fc;
      } else {
        // FP32 output: FP32 transcendentals whose small arguments are formed
        // from r^2 as an FP32 pair (about 44 bits, from the FP32-pair
        // positions: no FP64 instruction), keeping FP32 relative accuracy
        // near the cutoff:  1 - r/rc = (rc^2 - r^2) / (rc (rc + r)),
        // r - a = (r^2 - a^2) / (r + a), (1 + cos(pi r/rc))/2 = sin^2(pi u/2).
        const float2 r2 = bond_r2_pair(BP, ph, pl, i, j);
        const float rf = sqrtf(r2.x + r2.y);
        const float u = pair_diff(T.rc2, r2) / ((float)T.rcut * ((float)T.rcut + rf));
        const float sh = sinpif(0.5f * u);
        const float fc = u > 0.0f ? sh * sh : 0.0f;
        const float dr = pair_diff(r2, T.a2) / (rf + (float)T.a_cc);
        const float ex = expf(-(float)T.beta * dr * (float)T.inv_a);
        const float env = 1.0f + (float)T.gamma * (float)(ni + ncount[j] - 6) * (1.0f / 6.0f);
        t = (double)((float)T.pref[zic * 3 + zj] * ex * env * fc);
      }
    }
    val[e] = static_cast<valT>(t);
  }
  if (diag) diag[i] = static_cast<valT>(T.onsite[zic]);
}

}  // namespace
}  // namespace gputb

using namespace gputb;

extern "C" size_t tb_build_hamiltonian_teacher_workspace_size(int64_t n, int32_t precision) {
  if (n < 0) return 0;
  // the species-check word; for FP32 values also the FP32-pair positions
  return 256 + (precision == TB_F32 ? (size_t)n * 2 * sizeof(float4) : 0);
}

extern "C" tb_status tb_build_hamiltonian_teacher(const double *positions, const int32_t *species, int64_t n,
                                                  const double *box, const int32_t *pbc, const int64_t *slice_ptr,
                                                  const int32_t *col, const int32_t *cnt, const int32_t *ncount,
                                                  const double *hop_prefactor, const double *onsite, double a_cc,
                                                  double beta, double gamma, double rcut, int32_t precision,
                                                  void *val, void *diag, void *workspace, size_t workspace_bytes,
                                                  void *stream) {
  TB_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "tb_build_hamiltonian_teacher: bad n");
  TB_REQUIRE(positions && species && slice_ptr && cnt && ncount && hop_prefactor && onsite,
             "tb_build_hamiltonian_teacher: null pointer argument");
  TB_REQUIRE(precision == TB_F32 || precision == TB_F64, "tb_build_hamiltonian_teacher: bad precision");
  TB_REQUIRE(a_cc > 0.0 && rcut > 0.0, "tb_build_hamiltonian_teacher: need a_cc > 0 and rcut > 0");
  TB_REQUIRE(workspace && (reinterpret_cast<uintptr_t>(workspace) & 255) == 0,
             "tb_build_hamiltonian_teacher: need a 256-byte aligned workspace");
  if (workspace_bytes < tb_build_hamiltonian_teacher_workspace_size(n, precision))
    return fail(TB_ERR_WORKSPACE, "tb_build_hamiltonian_teacher: workspace too small (%zu < %zu)", workspace_bytes,
                tb_build_hamiltonian_teacher_workspace_size(n, precision));
  Box B;
  tb_status s = make_box(box, pbc, rcut, &B);
  if (s != TB_OK) return s;
  TeacherConst T;
  for (int k = 0; k < 9; ++k) T.pref[k] = hop_prefactor[k];
  for (int k = 0; k < 3; ++k) T.onsite[k] = onsite[k];
  T.a_cc = a_cc;
  T.inv_a = 1.0 / a_cc;
  T.beta = beta;
  T.gamma = gamma;
  T.rcut = rcut;
  auto split = [](double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
  };
  T.rc2 = split(rcut * rcut);
  T.a2 = split(a_cc * a_cc);
  T.n_species = 3;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int *flags = static_cast<int *>(workspace);
  TB_CUDA(cudaMemsetAsync(flags, 0, sizeof(int), st));
  const unsigned nb = (unsigned)((((n + 31) / 32) * 32 + 255) / 256);
  if (precision == TB_F32) {
    float4 *ph = reinterpret_cast<float4 *>(static_cast<unsigned char *>(workspace) + 256);
    float4 *pl = ph + n;
    pos_pair_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(positions, n, ph, pl);
    TB_CHECK_LAUNCH();
    teacher_kernel<float><<<nb, 256, 0, st>>>(positions, ph, pl, species, n, B, box_pair(B), T, slice_ptr, col, cnt,
                                              ncount, static_cast<float *>(val), static_cast<float *>(diag), flags);
  } else {
    teacher_kernel<double><<<nb, 256, 0, st>>>(positions, nullptr, nullptr, species, n, B, box_pair(B), T, slice_ptr,
                                               col, cnt, ncount, static_cast<double *>(val),
                                               static_cast<double *>(diag), flags);
  }
  TB_CHECK_LAUNCH();
  int h = 0;
  TB_CUDA(cudaMemcpyAsync(&h, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  TB_CUDA(cudaStreamSynchronize(st));
  if (h & 1) return fail(TB_ERR_INVALID_ARG, "tb_build_hamiltonian_teacher: species outside [0, 3)");
  return TB_OK;
}
