/*
 * gputb.h -- C ABI of the GB300 (sm_103a) GPUTB hot path.
 *
 * The library maps atomic structures to an orthogonal sparse tight-binding
 * Hamiltonian (Eq. 1 and Eq. 2 of arXiv 2509.06525, Sec. 3) and runs the
 * linear-scaling kernel polynomial method on it to obtain the density of
 * states (Eq. 4, Sec. 2.4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every array argument marked "device" is caller-owned device memory on
 *   the current CUDA device; "host" arrays are caller-owned host memory that
 *   is only read (or written where stated) during the call.  The library
 *   never frees caller memory and keeps no pointer after returning.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Work is enqueued on it.  Calls that must report a device-side
 *   condition (overflow, bounds violation) synchronise that stream before
 *   returning; this is stated per call.
 * - `workspace` / `workspace_bytes`: scratch device memory supplied by the
 *   caller, at least the size returned by the matching *_workspace_size
 *   query, 256-byte aligned.  Its contents on entry are ignored.
 * - Every call returns a tb_status; TB_OK is 0.  On failure tb_last_error()
 *   returns a message for the calling thread.  No call aborts the process.
 *
 * Sparse format (sliced ELL, slice height 32, "SELL-32")
 * -----------------------------------------------------
 * Rows are grouped in slices of 32 consecutive rows; n_slices = ceil(N/32).
 * slice_ptr (int64, device, n_slices + 1 entries) holds the element offset
 * of each slice; slice k has width w_k = (slice_ptr[k+1] - slice_ptr[k]) / 32
 * and stores its elements slot-major: element (row i, slot s) lives at
 *     slice_ptr[i / 32] + s * 32 + (i % 32),       0 <= s < w_(i/32).
 * col (int32) and the values share this layout.  Within a row the occupied
 * slots hold the neighbours j in ascending order; padding slots hold
 * col = i and value 0 (rows i >= N of the last slice hold col = 0).
 *
 * Boxes: box is 9 host doubles, row k = lattice vector a_k, in the lower-
 * triangular form a1 = (ax,0,0), a2 = (bx,by,0), a3 = (cx,cy,cz) with
 * ax, by, cz > 0.  pbc is 3 host int32 flags.  A periodic direction must have
 * a perpendicular width >= 2 rcut (else TB_ERR_BOX).
 */
#ifndef GPUTB_H
#define GPUTB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GPUTB_ABI_VERSION 1

#if defined(__GNUC__)
#define TB_API __attribute__((visibility("default")))
#else
#define TB_API
#endif

typedef int32_t tb_status;
#define TB_OK                 0
#define TB_ERR_INVALID_ARG    1   /* bad size, pointer, enum or layout      */
#define TB_ERR_CUDA           2   /* a CUDA runtime call failed              */
#define TB_ERR_WORKSPACE      3   /* workspace missing or too small          */
#define TB_ERR_BOX            4   /* periodic width < 2 rcut / bad box form  */
#define TB_ERR_ELL_OVERFLOW   5   /* a row has more neighbours than allowed  */
#define TB_ERR_BOUNDS         6   /* |mu_n| > 1 + 1e-6: spectrum outside [-1,1] after rescaling */
#define TB_ERR_NOT_FINITE     7   /* NaN/Inf met in an input or result       */

/* precision of Hamiltonian values and KPM vectors */
#define TB_F32 0
#define TB_F64 1

/* KPM damping kernels (Weisse et al., Rev. Mod. Phys. 78, 275 (2006)) */
#define TB_KERNEL_JACKSON 0
#define TB_KERNEL_LORENTZ 1
#define TB_KERNEL_NONE    2

/* Library ABI version (GPUTB_ABI_VERSION of the build). */
TB_API int32_t tb_abi_version(void);

/* Message describing the last failure on the calling thread ("" if none). */
TB_API const char *tb_last_error(void);

/* ---------------------------------------------------------------------
 * KPM moments (Sec. 2.4: Chebyshev expansion, KPM, SpMV, random phases).
 *
 * Computes, for r = 0..R-1 and n = 0..M-1,
 *     mu_r[r*M + n] = Re( sum_i conj(v0[i,r]) (T_n(H~) v0)[i,r] ) / N
 * with H~ = (H - b) / a, H = offdiag(col, val) + diag(diag), the random
 * phase vectors v0[i,r] = exp(2 pi i u(seed, r, i)) where
 *     u(seed, r, i) = (splitmix64(seed ^ splitmix64(r * 2^32 + i)) >> 11) * 2^-53
 * and splitmix64 is one output of SplitMix64 from state x (Steele, Lea &
 * Flood 2014).  T_n(H~) v0 uses the recursion v1 = H~ v0,
 * v_{n+1} = 2 H~ v_n - v_{n-1}.  Vector arithmetic is in `precision`
 * (TB_F32: complex FP32, TB_F64: complex FP64); every moment partial sum is
 * accumulated in FP64 and reduced in a fixed order (bitwise reproducible).
 *
 *   n            number of rows N (>= 1, < 2^31)
 *   slice_ptr    device int64 [ceil(N/32)+1]        SELL-32 slice offsets
 *   col          device int32 [slice_ptr[last]]     column indices
 *   val          device float/double (per precision) off-diagonal values H_ij
 *   diag         device float/double [N] onsite H_ii, or NULL for all zero
 *   a, b         rescaling H~ = (H - b)/a; a > 0
 *   M            moments (>= 2);  R  vectors: 1, 2, 4, 8, 16 or 32
 *   seed         random-phase seed
 *   mu_r         device double [R*M] output (vector r, moment n at r*M+n)
 *   workspace    >= kpm_moments_workspace_size(n, M, R, precision) bytes
 * Synchronises `stream`, then checks |mu_r| <= 1 + 1e-6 (TB_ERR_BOUNDS)
 * and finiteness (TB_ERR_NOT_FINITE).
 * ------------------------------------------------------------------- */
TB_API size_t kpm_moments_workspace_size(int64_t n, int32_t M, int32_t R, int32_t precision);

TB_API tb_status kpm_moments(int64_t n, const int64_t *slice_ptr, const int32_t *col,
                      const void *val, const void *diag, int32_t precision,
                      double a, double b, int32_t M, int32_t R, uint64_t seed,
                      double *mu_r, void *workspace, size_t workspace_bytes,
                      void *stream);

/* ---------------------------------------------------------------------
 * KPM density of states, Eq. 4, per orbital per eV (integrates to 1):
 *   rho(E_k) = [g_0 mu_0 + 2 sum_{n>=1} g_n mu_n T_n(x_k)] / (pi a sqrt(1-x_k^2))
 * with x_k = (E_k - b)/a, rho = 0 where |x_k| >= 1, mu_n the mean over the
 * R rows of mu_r, and g_n the damping kernel (Jackson: Weisse et al. 2006
 * Eq. 71; Lorentz: g_n = sinh(lambda(1-n/M))/sinh(lambda); none: g_n = 1).
 * Multiply by 2 (spin) and N/Omega for the (2/Omega) normalisation of Eq. 4.
 *
 *   mu_r     device double [R*M]   energy  device double [K]
 *   dos      device double [K] output
 * ------------------------------------------------------------------- */
TB_API tb_status kpm_dos(const double *mu_r, int32_t R, int32_t M, int32_t kernel,
                  double lambda, double a, double b, const double *energy,
                  int32_t K, double *dos, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GPUTB_H */
