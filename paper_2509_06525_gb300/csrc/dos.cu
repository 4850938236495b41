// KPM density of states, Eq. 4 of arXiv 2509.06525 (per orbital, per eV):
//   rho(E) = [g_0 mu_0 + 2 sum_{n>=1} g_n mu_n T_n(x)] / (pi a sqrt(1 - x^2)),
//   x = (E - b) / a, rho = 0 for |x| >= 1,
// with the Jackson / Lorentz damping of Weisse et al., RMP 78, 275 (2006).
//
// Each CTA first forms c_n = g_n mean_r(mu_r[., n]) (times 2 for n >= 1) in
// shared memory, then every thread sums the Chebyshev series for one energy
// with the three-term recurrence in FP64.  M * K is at most a few million
// terms, far below any roofline; the kernel exists so the whole path stays
// on the device.
#include <cmath>

#include "common.cuh"

namespace gputb {
namespace {

constexpr int kMaxDosM = 16384;

__global__ void dos_kernel(const double *__restrict__ mu_r, int R, int M, int kernel, double lambda, double a,
                           double b, const double *__restrict__ energy, int K, double *__restrict__ dos) {
  extern __shared__ double coef[];
  const double q = M_PI / (double)(M + 1);
  const double cot_q = cos(q) / sin(q);
  for (int n = threadIdx.x; n < M; n += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < R; ++r) s += mu_r[(int64_t)r * M + n];
    const double mu = s / (double)R;
    double g = 1.0;
    if (kernel == TB_KERNEL_JACKSON)
      g = ((double)(M - n + 1) * cos(q * n) + sin(q * n) * cot_q) / (double)(M + 1);
    else if (kernel == TB_KERNEL_LORENTZ)
      g = sinh(lambda * (1.0 - (double)n / (double)M)) / sinh(lambda);
    coef[n] = (n == 0 ? 1.0 : 2.0) * g * mu;
  }
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double x = (energy[k] - b) / a;
  if (!(fabs(x) < 1.0)) {
    dos[k] = 0.0;
    return;
  }
  double t0 = 1.0, t1 = x;
  double sum = coef[0] + (M > 1 ? coef[1] * x : 0.0);
  for (int n = 2; n < M; ++n) {
    const double t2 = 2.0 * x * t1 - t0;
    sum += coef[n] * t2;
    t0 = t1;
    t1 = t2;
  }
  dos[k] = sum / (M_PI * a * sqrt(1.0 - x * x));
}

}  // namespace
}  // namespace gputb

using namespace gputb;

extern "C" tb_status kpm_dos(const double *mu_r, int32_t R, int32_t M, int32_t kernel, double lambda, double a,
                             double b, const double *energy, int32_t K, double *dos, void *stream) {
  TB_REQUIRE(mu_r && energy && dos, "kpm_dos: null pointer argument");
  TB_REQUIRE(R >= 1 && M >= 1 && M <= kMaxDosM && K >= 0, "kpm_dos: bad sizes R=%d M=%d K=%d", R, M, K);
  TB_REQUIRE(kernel == TB_KERNEL_JACKSON || kernel == TB_KERNEL_LORENTZ || kernel == TB_KERNEL_NONE,
             "kpm_dos: bad kernel %d", kernel);
  TB_REQUIRE(a > 0.0 && std::isfinite(b), "kpm_dos: need a > 0");
  TB_REQUIRE(kernel != TB_KERNEL_LORENTZ || lambda > 0.0, "kpm_dos: Lorentz kernel needs lambda > 0");
  if (K == 0) return TB_OK;
  const size_t smem = (size_t)M * sizeof(double);
  TB_CUDA(cudaFuncSetAttribute(dos_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kMaxDosM * 8)));
  dos_kernel<<<(K + 255) / 256, 256, smem, static_cast<cudaStream_t>(stream)>>>(mu_r, R, M, kernel, lambda, a, b,
                                                                                  energy, K, dos);
  TB_CHECK_LAUNCH();
  return TB_OK;
}
