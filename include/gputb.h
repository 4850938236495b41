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
 * col = i and value 0 (rows i >= N of the last slice hold col = 0 and
 * value 0).
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

#define GPUTB_ABI_VERSION 9

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
#define TB_ERR_TIMEOUT        8   /* a bounded device-side wait gave up      */
#define TB_ERR_NOT_CONVERGED  9   /* an iteration stopped at its sweep limit */

/* precision of Hamiltonian values and KPM vectors */
#define TB_F32 0
#define TB_F64 1

/* how kpm_moments forms the moments */
#define TB_KPM_DIRECT   0   /* mu_n = Re<v0|v_n>/N, one step per moment           */
#define TB_KPM_DOUBLING 1   /* mu_2k = 2<v_k|v_k>/N - mu_0, mu_2k+1 = 2 Re<v_k|v_k+1>/N - mu_1:
                               about M/2 steps and no v0 stream (Weisse et al. 2006) */

/* KPM damping kernels (Weisse et al., Rev. Mod. Phys. 78, 275 (2006)) */
#define TB_KERNEL_JACKSON 0
#define TB_KERNEL_LORENTZ 1
#define TB_KERNEL_NONE    2

/* Library ABI version (GPUTB_ABI_VERSION of the build). */
TB_API int32_t tb_abi_version(void);

/* Message describing the last failure on the calling thread ("" if none). */
TB_API const char *tb_last_error(void);

/* Number of kernel launches this process has issued through the library. */
TB_API int64_t tb_launch_count(void);

/* Host <-> device boundary (no counterpart in the paper).  Every other call
 * takes device arrays; host inputs (positions, species) enter through
 * tb_copy_to_device and results (moments, DOS) leave through
 * tb_copy_to_host, each one cudaMemcpyAsync on `stream` (page-locked host
 * memory makes them asynchronous DMA transfers).  tb_copy_to_host
 * synchronises `stream` before returning, so the host array is filled. */
TB_API tb_status tb_copy_to_device(void *dst_device, const void *src_host, size_t bytes, void *stream);
TB_API tb_status tb_copy_to_host(void *dst_host, const void *src_device, size_t bytes, void *stream);

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
 * v_{n+1} = 2 H~ v_n - v_{n-1}.  With mode TB_KPM_DOUBLING the same moments
 * come from the product identities T_2k = 2 T_k^2 - T_0 and
 * T_2k+1 = 2 T_k T_k+1 - T_1 applied to the vectors (equal in exact
 * arithmetic), which needs only about M/2 steps.  Vector arithmetic is in `precision`
 * (TB_F32: complex FP32, TB_F64: complex FP64); every moment partial sum is
 * accumulated in FP64 and reduced in a fixed order (bitwise reproducible).
 *
 *   n            number of rows N (>= 1, < 2^31)
 *   slice_ptr    device int64 [ceil(N/32)+1]        SELL-32 slice offsets
 *   col          device int32 [slice_ptr[last]]     column indices
 *   val          device float/double (per precision) off-diagonal values H_ij
 *                (col and val may be NULL when every slice has width 0)
 *   diag         device float/double [N] onsite H_ii, or NULL for all zero
 *   a, b         rescaling H~ = (H - b)/a; a > 0
 *   M            moments (>= 2);  R  vectors: 1, 2, 4, 8, 16 or 32
 *   seed         random-phase seed
 *   first_vector index of this call's first random vector (0 .. 2^31):
 *                vector r uses u(seed, first_vector + r, i), so calls (or
 *                ranks) holding disjoint index ranges compute members of one
 *                ensemble, identical to one call over the union
 *   mode         TB_KPM_DIRECT or TB_KPM_DOUBLING
 *   mu_r         device double [R*M] output (vector r, moment n at r*M+n)
 *   workspace    >= kpm_moments_workspace_size(n, M, R, precision) bytes
 *   step_ms      host double or NULL: if given, receives the CUDA-event time
 *                (ms) of the M-1 Chebyshev-step launches on `stream`
 * Synchronises `stream`, then checks |mu_r| <= 1 + 1e-6 (TB_ERR_BOUNDS)
 * and finiteness (TB_ERR_NOT_FINITE).  The pipelined step kernel bounds
 * every wait on its copy barriers and reports TB_ERR_TIMEOUT if one gives
 * up.  col and val must be 16-byte aligned (diag too for shapes of kind 2).
 * ------------------------------------------------------------------- */
TB_API size_t kpm_moments_workspace_size(int64_t n, int32_t M, int32_t R, int32_t precision);

/* ---------------------------------------------------------------------
 * Step shapes and their autotuner (no counterpart in the paper: launch
 * configuration of this library's Chebyshev-step kernel).
 *
 * For each (R, precision) the library carries a fixed list of compiled
 * launch shapes of the Chebyshev step; entry 0 is the default.  A shape is
 * the kernel family (direct loads, or a bulk-copy ring of `stages` tiles in
 * shared memory), the complex numbers each thread moves (R divided by it =
 * threads per row), the resident CTAs per SM its register budget is sized
 * for, and the rows one CTA processes per tile.  Every shape computes the
 * same moments up to the grouping of the FP64 partial sums (differences of
 * a few ulps), and each shape on its own is bitwise reproducible.
 *
 * kpm_moments, kpm_moments_noalloc, kpm_moments_batched and lsqt_vac use,
 * for (precision, R, mode, n): the shape forced for every size (n = 0 entry)
 * if one is set, else the entry of n's size class floor(log2 n), else 0.
 * The table is process-wide and guarded by a mutex; workspace sizes cover
 * every shape, so a workspace queried once stays valid when the table
 * changes.
 * ------------------------------------------------------------------- */
typedef struct {
  int32_t pipelined;            /* 0: direct loads; 1: bulk-copy ring of col, val
                                   and vector rows; 2: ring that also stages the
                                   slice offsets and the diagonal; 3: banded
                                   step (x bands staged, needs the band plan,
                                   which kpm_moments builds in its workspace) */
  int32_t complex_per_thread;   /* complex numbers per thread (R / threads per row) */
  int32_t stages;               /* ring depth (0 for direct loads)           */
  int32_t min_blocks;           /* resident CTAs per SM of the register budget */
  int32_t rows_per_tile;        /* rows a CTA processes per tile             */
  int32_t rows_per_thread;      /* rows each thread takes per tile           */
  int32_t staged_vectors;       /* 1: v_{n-1} (and v0) rows go through the ring */
  int32_t options;              /* ring (1): 1 = 12-slot body for slices at most
                                   12 wide; banded (3): 1 = no CTA barrier per
                                   tile (stages released per warp)          */
  int32_t band_rows;            /* banded (3): x rows a stage holds          */
} tb_step_shape;

/* Number of shapes for (R, precision); 0 if R is unsupported. */
TB_API int32_t tb_kpm_shape_count(int32_t R, int32_t precision);
/* Description of shape `shape`; TB_ERR_INVALID_ARG if out of range. */
TB_API tb_status tb_kpm_shape_info(int32_t R, int32_t precision, int32_t shape, tb_step_shape *out);
/* Set the table entry of n's size class (n > 0) or the forced entry (n = 0)
 * for mode TB_KPM_DIRECT, TB_KPM_DOUBLING or both (mode = -1); shape = -1
 * removes the entry. */
TB_API tb_status tb_kpm_set_shape(int64_t n, int32_t R, int32_t precision, int32_t mode, int32_t shape);
/* Remove every entry (all calls use shape 0 again). */
TB_API tb_status tb_kpm_clear_shapes(void);
/* The shape a call with these arguments would use; -1 if unsupported. */
TB_API int32_t tb_kpm_get_shape(int64_t n, int32_t R, int32_t precision, int32_t mode);
/* CTAs of one Chebyshev-step launch of `shape` over n rows in `mode` (the
 * occupancy-limited grid: min(tiles, resident CTAs per SM x SMs)); each CTA
 * processes ceil(tiles / grid) or fewer tiles of rows_per_tile rows.  Queries
 * the current device; -1 on bad arguments or a failed query. */
TB_API int32_t tb_kpm_shape_grid(int64_t n, int32_t R, int32_t precision, int32_t mode, int32_t shape);

/* Autotuner: on the caller's matrix (arguments as kpm_moments), draws the
 * random phases, forms v1 with shape 0, then for every shape of
 * (R, precision) runs 2 warm-up and `reps` timed steps of the recursion in
 * `mode` (the same kernels, operands and in-place update as kpm_moments;
 * CUDA events on `stream`).  ms_per_step (host float [ms_capacity] or NULL)
 * receives the mean time per step of each shape; *best_shape the fastest,
 * which is also stored as the table entry of n's size class for this mode.
 *   reps        1 .. 10000
 *   workspace   >= kpm_moments_workspace_size(n, 2, R, precision) bytes
 * Synchronises `stream`; TB_ERR_TIMEOUT if a pipeline wait gave up. */
TB_API tb_status tb_kpm_autotune(int64_t n, const int64_t *slice_ptr, const int32_t *col,
                                 const void *val, const void *diag, int32_t precision, double a,
                                 double b, int32_t R, int32_t mode, int32_t reps, void *workspace,
                                 size_t workspace_bytes, void *stream, int32_t *best_shape,
                                 float *ms_per_step, int32_t ms_capacity);

TB_API tb_status kpm_moments(int64_t n, const int64_t *slice_ptr, const int32_t *col,
                      const void *val, const void *diag, int32_t precision,
                      double a, double b, int32_t M, int32_t R, uint64_t seed,
                      int64_t first_vector, int32_t mode, double *mu_r, void *workspace,
                      size_t workspace_bytes, void *stream, double *step_ms);

/* ---------------------------------------------------------------------
 * kpm_moments without any device allocation (no counterpart in the paper;
 * an interface convenience of this library).
 *
 * For callers that cannot allocate device memory where they need the
 * moments: code inside a framework that owns the device memory pool,
 * latency-critical loops where cudaMalloc would synchronise the device, or
 * plug-ins that are handed only their input and output buffers.  Same
 * arguments, results and checks as kpm_moments in TB_KPM_DIRECT mode, minus
 * the mode, the workspace and the timing output: the scratch lives in a static 32 MiB device array inside the
 * library, which every GPU that loads the library keeps until the process
 * exits.  Sizes whose kpm_moments_workspace_size exceeds 32 MiB are rejected
 * with TB_ERR_WORKSPACE (use kpm_moments with a caller workspace instead).
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and every call
 * overwrites it: calls whose GPU work may overlap (other streams, other host
 * threads on the same device) race and must be serialised by the caller.
 * No cudaMalloc, cudaFree or other allocating routine is called.
 * Synchronises `stream`.
 * ------------------------------------------------------------------- */
TB_API tb_status kpm_moments_noalloc(int64_t n, const int64_t *slice_ptr, const int32_t *col,
                                     const void *val, const void *diag, int32_t precision,
                                     double a, double b, int32_t M, int32_t R, uint64_t seed,
                                     double *mu_r, void *stream);

/* ---------------------------------------------------------------------
 * Batched KPM over many uneven snapshots (multi-frame averaging of the
 * LSQT calculation, Sec. 2.4), one CUDA-graph launch for all of them.
 *
 * Snapshot s (0 <= s < n_snap) is a SELL-32 Hamiltonian with n_rows[s]
 * rows given by the device pointers slice_ptr[s], col[s], val[s], diag[s]
 * (diag[s] may be NULL; the pointer arrays themselves are host arrays), with
 * its own rescaling (a[s], b[s]) (host arrays).  Its moments are those of
 * kpm_moments(H_s, a[s], b[s], M, R, seed + s, mode): random phases of
 * snapshot s use seed + s and the snapshot's own row numbers.  The call
 * folds every (a[s], b[s]) into a block-diagonal copy of the matrices in the
 * workspace (snapshots padded to 256-row tiles), runs the shared Chebyshev
 * step kernels with one moment partial per row block, and captures the
 * whole recursion as a CUDA graph launched on `stream`.  The workspace-size
 * query reads each snapshot's element count from its slice_ptr and
 * synchronises `stream`.
 *
 * The graph holds the fold of every snapshot, the band plan (banded step
 * shapes), the random phases, every Chebyshev step and the reduction.  The
 * library keeps the instantiated graph of the last call and launches it
 * again while the next call has the same device, pointers, sizes, element
 * counts, (a, b), M, R, seed, mode, step shape and workspace; any
 * difference captures a new one (the first call of a layout pays the
 * capture and instantiation).  Calls are serialised by a mutex.
 *   mu         device double [n_snap][R][M] output
 *   graph_ms   host double or NULL: CUDA-event time of the graph launch
 *              (fold and recursion; not the capture)
 * Synchronises `stream`; TB_ERR_BOUNDS / TB_ERR_NOT_FINITE as kpm_moments.
 * ------------------------------------------------------------------- */
TB_API size_t kpm_moments_batched_workspace_size(int32_t n_snap, const int64_t *const *slice_ptr,
                                                 const int64_t *n_rows, int32_t M, int32_t R,
                                                 int32_t precision, void *stream);

TB_API tb_status kpm_moments_batched(int32_t n_snap, const int64_t *n_rows,
                                     const int64_t *const *slice_ptr, const int32_t *const *col,
                                     const void *const *val, const void *const *diag,
                                     int32_t precision, const double *a, const double *b,
                                     int32_t M, int32_t R, uint64_t seed, int32_t mode, double *mu,
                                     void *workspace, size_t workspace_bytes, void *stream,
                                     double *graph_ms);

/* Autotuner of the batched path (no counterpart in the paper): folds the
 * batch as kpm_moments_batched does (same arguments and workspace), then
 * times every step shape on the folded block-diagonal matrix as
 * tb_kpm_autotune does and stores the fastest as the table entry of the
 * batch's padded row count.  Synchronises `stream`. */
TB_API tb_status kpm_moments_batched_autotune(int32_t n_snap, const int64_t *n_rows,
                                              const int64_t *const *slice_ptr,
                                              const int32_t *const *col, const void *const *val,
                                              const void *const *diag, int32_t precision,
                                              const double *a, const double *b, int32_t R,
                                              int32_t mode, int32_t reps, void *workspace,
                                              size_t workspace_bytes, void *stream,
                                              int32_t *best_shape, float *ms_per_step,
                                              int32_t ms_capacity);

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


/* Test hook (no counterpart in the paper): runs the bounded wait of the
 * pipelined step (an mbarrier phase) on a phase that nothing completes, with
 * a limit of `polls` polls.  Returns TB_ERR_TIMEOUT when the wait gave up
 * (the expected outcome; the context stays usable), TB_OK if it completed.
 *   workspace   device, >= 256 bytes (zeroed by the call)
 * Synchronises `stream`. */
TB_API tb_status tb_debug_wait_timeout(int64_t polls, void *workspace, size_t workspace_bytes,
                                       void *stream);

/* ---------------------------------------------------------------------
 * Velocity-autocorrelation conductivity, Eq. 3 (sigma) of Sec. 2.4:
 *   sigma(E, t) = (2 e^2 / Omega) int_0^t Tr[delta(E - H) Re(V V(tau))] dtau,
 *   V(tau) = exp(i H tau/hbar) V exp(-i H tau/hbar),  V = (i/hbar)[H, X].
 *
 * tb_velocity_values: the real SELL values of V / (i/hbar) along the unit
 * direction e: vval_ij = H_ij (d_ij . e), d_ij the minimum-image bond vector
 * (same pattern as H; padding and phantom rows 0).
 *   positions   device double [N][3];  box/pbc/rcut as tb_build_neighbors
 *   val         device float/double SELL values of H;  vval  same layout, output
 *   direction   host double [3]
 *
 * lsqt_vac: per-vector VAC moments
 *   mu_out[j][r][n] = Re <V phi_L(t_j)| T_n(H~) |phi_R(t_j)> / N,  t_j = j dt,
 * with phi_L(0) = V phi_r, phi_R(0) = phi_r, phi_r the random-phase vector
 * first_vector + r of kpm_moments, both propagated by U(dt) = exp(-i H dt/hbar)
 * (Chebyshev-Bessel series of exp(-i (a dt/hbar) H~) times exp(-i b dt/hbar),
 * cut where |J_k| < 1e-17).  hbar = 0.6582119569 eV fs; H in eV, positions
 * in Angstrom, dt in fs, so the moments are in Angstrom^2/fs^2.
 *   n, slice_ptr, col, val, diag, precision, a, b, M, R, seed: as kpm_moments
 *                (R: 1, 2, 4, 8 or 16; a dt / hbar <= 200)
 *   vval         device, from tb_velocity_values
 *   n_steps      time steps (n_steps + 1 time points, t_0 = 0)
 *   mu_out       device double [(n_steps + 1) * R * M]
 *   ms_out       host double or NULL: CUDA-event time of the whole loop (ms)
 * Synchronises `stream`; TB_ERR_NOT_FINITE for non-finite moments,
 * TB_ERR_TIMEOUT if a bounded pipeline wait gives up.
 *
 * lsqt_correlation: per-orbital C(E_k, t_j) = (1/N) Re Tr[delta(E - H) V V(t_j)]
 * (the damped Chebyshev series of kpm_dos applied to the vector-averaged
 * moments) and S(E_k, t_j) = int_0^{t_j} C dtau by the trapezoid rule
 * (S(E, 0) = 0); sigma(E, t) = (2 e^2 N / Omega) S(E, t).
 *   mu           device double [n_times][R][M] (lsqt_vac output)
 *   energy       device double [K];  corr, sigma  device double [n_times][K]
 *                (sigma may be NULL);  coef_ws device double [n_times * M]
 * ------------------------------------------------------------------- */
TB_API tb_status tb_velocity_values(const double *positions, int64_t n, const double *box,
                                    const int32_t *pbc, double rcut, const int64_t *slice_ptr,
                                    const int32_t *col, const void *val, int32_t precision,
                                    const double *direction, void *vval, void *stream);

TB_API size_t lsqt_vac_workspace_size(int64_t n, int32_t M, int32_t R, int32_t precision);

TB_API tb_status lsqt_vac(int64_t n, const int64_t *slice_ptr, const int32_t *col,
                          const void *val, const void *diag, const void *vval, int32_t precision,
                          double a, double b, int32_t M, int32_t R, uint64_t seed,
                          int64_t first_vector, int32_t n_steps, double dt_fs, double *mu_out,
                          void *workspace, size_t workspace_bytes, void *stream, double *ms_out);

TB_API tb_status lsqt_correlation(const double *mu, int32_t n_times, int32_t R, int32_t M,
                                  int32_t kernel, double lambda, double a, double b,
                                  const double *energy, int32_t K, double dt_fs, double *corr,
                                  double *sigma, double *coef_ws, void *stream);

/* ---------------------------------------------------------------------
 * Multi-orbital (s, p, d) Slater-Koster Hamiltonian, matrix-free (the SK
 * angular factors of Sec. 3; orbitals per atom: s, p_x, p_y, p_z, d_xy,
 * d_yz, d_zx, d_x2-y2, d_3z2-r2, orbital index 9 i + a).  Each SELL element
 * of the neighbour structure keeps the compressed SK form of its bond --
 * direction cosines l, m, n of d_ij = r_j - r_i and the ten two-centre
 * integrals V_k(r) = v0[k] exp(-beta (r/a_cc - 1)) f_c(r) in the order
 * ss_sigma, sp_sigma, pp_sigma, pp_pi, sd_sigma, pd_sigma, pd_pi, dd_sigma,
 * dd_pi, dd_delta -- and every use rebuilds the 9 x 9 block from the
 * closed-form Slater-Koster table.
 *
 * tb_sk_geometry: geom = device float [13][total] planes (l, m, n, V_0..V_9;
 *   zero for padding slots and phantom rows); positions/box/pbc/rcut as
 *   tb_build_neighbors; v0 host double [10].  Synchronises `stream`.
 * tb_sk_bounds: Gershgorin enclosure of the spectrum (onsite host double [3]:
 *   E_s, E_p, E_d) -> bounds_out host double [4] = {E_min, E_max, a, b} with
 *   a = (E_max - E_min)/(2 - 0.01), b = midpoint; workspace >= 4 KB +
 *   16 bytes per CTA (use sk_kpm_workspace_size).  Synchronises `stream`.
 * sk_kpm_moments: KPM moments of the 9N-orbital H for random-phase vector
 *   first_vector (orbital index as the row: u(seed, first_vector, 9 i + a)),
 *   moment doubling, complex FP32 vectors, FP64 sums:
 *   mu_out device double [M] = Re <v0|T_n(H~)|v0> / (9N).  Checks |mu| <= 1
 *   + 1e-6 (TB_ERR_BOUNDS) and finiteness.  ms_out as lsqt_vac.
 * ------------------------------------------------------------------- */
TB_API tb_status tb_sk_geometry(const double *positions, int64_t n, const double *box,
                                const int32_t *pbc, double rcut, const int64_t *slice_ptr,
                                const int32_t *col, int64_t total, const double *v0, double a_cc,
                                double beta, float *geom, void *stream);

TB_API tb_status tb_sk_bounds(int64_t n, const int64_t *slice_ptr, const int32_t *col,
                              const float *geom, int64_t total, const double *onsite,
                              double *bounds_out, void *workspace, size_t workspace_bytes,
                              void *stream);

TB_API size_t sk_kpm_workspace_size(int64_t n, int32_t M);

TB_API tb_status sk_kpm_moments(int64_t n, const int64_t *slice_ptr, const int32_t *col,
                                const float *geom, int64_t total, const double *onsite, double a,
                                double b, int32_t M, uint64_t seed, int64_t first_vector,
                                double *mu_out, void *workspace, size_t workspace_bytes,
                                void *stream, double *ms_out);

/* ---------------------------------------------------------------------
 * Neighbour lists N(i) of Eq. 1 (Sec. 3): every j != i with a periodic
 * image closer than rcut, found with a device cell list and written as the
 * SELL-32 column array of the Hamiltonian (row i's neighbours ascending,
 * padding col = i).  Membership is decided in FP64 as
 *   ((dx*dx) + (dy*dy)) + (dz*dz) < rcut*rcut
 * with each operation rounded separately, d being the minimum-image
 * displacement reduced along a3, then a2, then a1.  Non-periodic directions
 * are not binned (one cell layer), which suits sheets and slabs.
 *
 *   positions   device double [N][3] (Angstrom)
 *   r_count     also count n_i = #{j: r_ij < r_count} into ncount (<= 0: skip)
 *   max_width   maximum slots per row (1..64); a row with more neighbours
 *               returns TB_ERR_ELL_OVERFLOW
 *   slice_ptr   device int64 [ceil(N/32)+1] output; slice width = the
 *               largest neighbour count among its 32 rows
 *   col         device int32 [col_capacity] output; N' = ceil(N/32)*32*max_width
 *               elements always suffice.  If the structure needs more than
 *               col_capacity, TB_ERR_ELL_OVERFLOW is returned, *total_out
 *               holds the size needed and col is not written.
 *   cnt         device int32 [N] output: neighbours per row
 *   ncount      device int32 [N] output or NULL
 *   total_out   host int64: number of SELL elements (slice_ptr[last])
 * Synchronises `stream`.  Positions must be finite (TB_ERR_NOT_FINITE), and
 * every wrapped coordinate within 2^20 * rcut of the origin
 * (TB_ERR_INVALID_ARG): the FP32 pair screen's error bound assumes it.
 * The workspace size (0 for an invalid box, rcut or max_width) depends on
 * max_width: the search keeps every row's sorted list once.
 * ------------------------------------------------------------------- */
TB_API size_t tb_neighbors_workspace_size(int64_t n, const double *box, const int32_t *pbc, double rcut,
                                          int32_t max_width);

TB_API tb_status tb_build_neighbors(const double *positions, int64_t n, const double *box,
                                    const int32_t *pbc, double rcut, double r_count,
                                    int32_t max_width, int64_t *slice_ptr, int32_t *col,
                                    int64_t col_capacity, int32_t *cnt, int32_t *ncount,
                                    int64_t *total_out, void *workspace, size_t workspace_bytes,
                                    void *stream);

/* ---------------------------------------------------------------------
 * Teacher Hamiltonian (analytic environment-dependent pz model, form of
 * Eq. 1; it replaces the DFT labels of Sec. 2.3):
 *   t_ij  = P[Z_i][Z_j] exp(-beta (r_ij/a_cc - 1)) (1 + gamma (n_i+n_j-6)/6) f_c(r_ij)
 *   f_c(r) = (1 + cos(pi r/rcut))/2 for r < rcut, else 0;  eps_i = onsite[Z_i]
 * evaluated from FP64 distances (exp and cos in `precision`) and stored in
 * `precision` into the SELL-32 layout of
 * (slice_ptr, col) from tb_build_neighbors (same positions and box).
 *
 *   species        device int32 [N], values 0..2 (else TB_ERR_INVALID_ARG)
 *   cnt, ncount    device int32 [N] from tb_build_neighbors (r_count = 1.8 A)
 *   hop_prefactor  host double [3][3] P (eV);  onsite  host double [3] (eV)
 *   val            device float/double [slice_ptr[last]] output
 *   diag           device float/double [N] output (onsite), or NULL
 *   workspace      device, 256-byte aligned, at least
 *                  tb_build_hamiltonian_teacher_workspace_size(n, precision)
 *                  bytes (the species check; for FP32 values also the
 *                  positions split into FP32 pairs, from which the bond
 *                  lengths are formed: r^2 to about 44 bits)
 * Synchronises `stream`.
 * ------------------------------------------------------------------- */
TB_API size_t tb_build_hamiltonian_teacher_workspace_size(int64_t n, int32_t precision);

TB_API tb_status tb_build_hamiltonian_teacher(const double *positions, const int32_t *species, int64_t n,
                                              const double *box, const int32_t *pbc,
                                              const int64_t *slice_ptr, const int32_t *col,
                                              const int32_t *cnt, const int32_t *ncount,
                                              const double *hop_prefactor, const double *onsite,
                                              double a_cc, double beta, double gamma, double rcut,
                                              int32_t precision, void *val, void *diag, void *workspace,
                                              size_t workspace_bytes, void *stream);

/* ---------------------------------------------------------------------
 * FP64 spectral bounds for the Chebyshev rescaling of Sec. 2.4.
 * Gershgorin enclosure [G_min, G_max]; `lanczos_steps` Lanczos steps (FP64,
 * no reorthogonalisation, start q_i = u(seed, 0, i) - 1/2 normalised, u as in
 * kpm_moments); Ritz extremes theta by Sturm multisection; then
 *   delta = 0.01 (theta_max - theta_min),
 *   E_max = min(G_max, theta_max + delta), E_min = max(G_min, theta_min - delta),
 *   a = (E_max - E_min)/(2 - 0.01), b = (E_max + E_min)/2.
 *   bounds_out  host double[8]: E_min, E_max, a, b, theta_min, theta_max, G_min, G_max
 * Synchronises `stream`.
 * ------------------------------------------------------------------- */
TB_API size_t tb_spectral_bounds_workspace_size(int64_t n, int32_t lanczos_steps);

TB_API tb_status tb_spectral_bounds(int64_t n, const int64_t *slice_ptr, const int32_t *col,
                                    const void *val, const void *diag, int32_t precision,
                                    int32_t lanczos_steps, uint64_t seed, double *bounds_out,
                                    void *workspace, size_t workspace_bytes, void *stream);

/* =====================================================================
 * Learned Hamiltonian (Sec. 3, Eq. 2; training per Sec. 2.1 and Eq. 3)
 *
 * Descriptors:  f_k(r) = (T_k(2(r/rcut - 1)^2 - 1) + 1)/2 f_c(r), k = 0..7,
 *               f_c(r) = (1 + cos(pi r/rcut))/2 (r < rcut);
 *               C_n(r_ij) = sum_k c[Z_i][Z_j][n][k] f_k(r_ij);
 *               v_i = sum_{j in N(i)} C(r_ij).
 * Edge input:   x_ij = [C(r_ij), v_i, v_j, C(r_ij)*(v_i + v_j)] (32 floats);
 *               xn = (x - mean) * inv_std.
 * Network:      y = W3 silu(W2 silu(W1 xn + b1) + b2) + b3, 32-64-64-2,
 *               BF16 weights and activations on tensor cores, FP32
 *               accumulation, FP32 master parameters.
 * Hamiltonian:  H_ij = (y0(i->j) + y0(j->i))/2, eps_i = eps0[Z_i] + sum_j y1(i->j).
 *
 * Parameter vector (FP32, 6402 floats, caller-owned, device):
 *   W1 [64][32] @0, b1 [64] @2048, W2 [64][64] @2112, b2 [64] @6208,
 *   W3 [2][64] @6272, b3 [2] @6400   (row-major [out][in]).
 * BF16 weight copy (6272 bf16): W1 @0, W2 @2048, W3 @6144.
 * cmix: device float [3][3][8][8];  v: device float [N][8].
 * Edge arrays (x, y, dy, t_hop) follow the SELL-32 element order of the
 * neighbour structure; padding elements hold zeros and are ignored.
 * ===================================================================== */

/* v_i for every atom (device float [N][8]). */
TB_API tb_status tb_compute_descriptors(const double *positions, const int32_t *species, int64_t n,
                                        const double *box, const int32_t *pbc, double rcut,
                                        const int64_t *slice_ptr, const int32_t *col, const int32_t *cnt,
                                        const float *cmix, float *v, void *stream);

/* Edge inputs of every SELL element: x_raw (device float [total][32], may be
 * NULL) and/or x_bf16 (device bf16 [total][32], normalised with mean/inv_std
 * (device float [32]) when both are given, else raw; may be NULL). */
TB_API tb_status tb_edge_features(const double *positions, const int32_t *species, int64_t n,
                                  const double *box, const int32_t *pbc, double rcut,
                                  const int64_t *slice_ptr, const int32_t *col, const int32_t *cnt,
                                  const float *cmix, const float *v, const float *mean,
                                  const float *inv_std, float *x_raw, void *x_bf16, void *stream);

/* Per-feature mean and standard deviation (population) of x_raw over the
 * real (non-padding) elements of rows 0..n-1, accumulated in FP64, and,
 * when inv_std (device float [32]) is given, the input normalisation
 *   inv_std[f] = mask[f] / max(std[f], 1e-6)
 * with mask (device float [32], may be NULL = all ones) switching features
 * off.  workspace >= 96 * 8 * 4 * (SM count) bytes. */
TB_API tb_status tb_feature_stats(const float *x_raw, int64_t n, const int64_t *slice_ptr,
                                  const int32_t *cnt, float *mean, float *stdv, float *inv_std,
                                  const float *mask, void *workspace, size_t workspace_bytes,
                                  void *stream);

/* inv_std[f] = mask[f] / max(stdv[f], 1e-6) for f < n (device float arrays;
 * mask may be NULL): the normalisation of tb_feature_stats for a caller's
 * own standard deviations. */
TB_API tb_status tb_inverse_std(const float *stdv, const float *mask, float *inv_std, int32_t n,
                                void *stream);

/* Workspace bytes of tb_mlp_backward for n_edges edges. */
TB_API size_t tb_mlp_workspace_size(int64_t n_edges);

/* y (device float [n_edges][2]) = MLP(x_bf16 [n_edges][32]). */
TB_API tb_status tb_mlp_forward(int64_t n_edges, const void *x_bf16, const void *w_bf16,
                                const float *params, float *y, void *stream);

/* grad (device float [6402]) = sum over edges of dL/dparams given dL/dy
 * (device float [n_edges][2]); the forward pass is recomputed.  Per-CTA
 * partial gradients are summed in a fixed order (reproducible). */
TB_API tb_status tb_mlp_backward(int64_t n_edges, const void *x_bf16, const void *w_bf16,
                                 const float *params, const float *dy, float *grad, void *workspace,
                                 size_t workspace_bytes, void *stream);

/* Loss of the form of Eq. 3 on the Hamiltonian of rows [row_begin, row_end)
 * (row_begin a multiple of 32):
 *   D = {y0(e) - t_hop(e) for the real elements e of those rows}
 *       U {eps0[Z_i] + sum_e y1(e) - eps_target(i)},  n = |D|,
 *   L = (sum|D|/n)^2 + sum D^2/n.
 * Writes dL/dy into dy for every element of those rows (0 for padding) and
 * stats (device double[4]) = {sum|D|/n, sum D^2/n, n, L}.
 * workspace >= 3 * 8 * 2 * (SM count) bytes. */
TB_API tb_status tb_mlp_loss(int64_t row_begin, int64_t row_end, const int64_t *slice_ptr,
                             const int32_t *cnt, const float *y, const float *t_hop,
                             const float *eps_target, const int32_t *species, const float *eps0,
                             float *dy, double *stats, void *workspace, size_t workspace_bytes,
                             void *stream);

/* One AdamW step (decoupled weight decay, bias-corrected moments; step >= 1)
 * on the FP32 parameters; refreshes the BF16 weight copy. */
TB_API tb_status tb_adamw_step(float *params, const float *grad, float *m, float *v, int64_t step,
                               double lr, double beta1, double beta2, double eps,
                               double weight_decay, void *w_bf16, void *stream);

/* BF16 weight copy from the FP32 parameters. */
TB_API tb_status tb_mlp_pack_weights(const float *params, void *w_bf16, void *stream);

/* Tuning hook for the forward pass of tb_build_hamiltonian: 0 = 5th-
 * generation tensor cores (tcgen05, accumulators in TMEM; default; bond
 * lengths from the positions split into FP32 pairs), 1 = mma.sync tiles
 * (bond lengths from FP64 coordinate differences).  Both compute the same
 * MLP in BF16 with FP32 accumulation (sums in a different order).
 * Process-wide. */
TB_API tb_status tb_mlp_set_variant(int32_t variant);

/* Workspace bytes of tb_build_hamiltonian for n atoms and total_elements
 * SELL elements (the two network outputs per element, status words and the
 * FP32-pair positions). */
TB_API size_t tb_build_hamiltonian_workspace_size(int64_t n, int64_t total_elements);

/* Learned Hamiltonian in SELL-32: val (device, `precision`, [total]) and
 * diag (device [N] or NULL).  v from tb_compute_descriptors on the same
 * structure; mean/inv_std may be NULL (no normalisation); eps0 device
 * float [3].  Synchronises `stream`; TB_ERR_INVALID_ARG if the neighbour
 * relation is not symmetric. */
TB_API tb_status tb_build_hamiltonian(const double *positions, const int32_t *species, int64_t n,
                                      const double *box, const int32_t *pbc, double rcut,
                                      const int64_t *slice_ptr, const int32_t *col, const int32_t *cnt,
                                      int64_t total_elements, const float *cmix, const float *v,
                                      const float *mean, const float *inv_std, const void *w_bf16,
                                      const float *params, const float *eps0, int32_t precision,
                                      void *val, void *diag, void *workspace, size_t workspace_bytes,
                                      void *stream);

/* ====================================================================
 * Environment network and band-energy training (Eq. 2 edge feature, the
 * SK form H_ij = sum_lambda MLP_lambda(e_ij) P_lambda(r_ij_hat) and the
 * onsite H_ii = MLP_alpha(v_i) of Sec. 3, the band loss of Eq. 3), for one
 * pz orbital per atom:
 *   u_ij = v_i + v_j   (= sum_{k in N(i)} C(r_ik) + sum_{l in N(j)} C(r_jl))
 *   m = MLP_e(u): 8 -> 32 (SiLU) -> 8;  e_ij = C(r_ij) * m  (elementwise)
 *   y = MLP_lambda(e): 8 -> 32 (SiLU) -> 32 (SiLU) -> 2  (sigma, pi)
 *   t_ij = y_sigma n_z^2 + y_pi (1 - n_z^2),  n_z = d_z / r
 *   eps_i = eps0[Z_i] + MLP_alpha(v_i)[Z_i]: 8 -> 32 (SiLU) -> 3
 * SiLU(z) = z / (1 + e^{-z}).  The mixing c^{Z_i Z_j} must be symmetric in
 * the species pair for H to be symmetric (u, r and n_z^2 are).
 *
 * Parameters: one device float vector [TB_ENV_NPARAM] in the order
 *   We1 [32][8], be1 [32], We2 [8][32], be2 [8],
 *   Wh1 [32][8], bh1 [32], Wh2 [32][32], bh2 [32], Wh3 [2][32], bh3 [2],
 *   Wo1 [32][8], bo1 [32], Wo2 [3][32], bo2 [3]   (weights [out][in]).
 * Bond inputs ("feat"): device float [total][TB_ENV_NFEAT] in SELL element
 * order: C[8], u[8], n_z^2, d[3] (bond vector r_j + T - r_i, Angstrom).
 * ==================================================================== */
#define TB_ENV_NPARAM 2349
#define TB_ENV_NFEAT 20

/* Bond inputs of every real SELL element of one structure (v from
 * tb_compute_descriptors with the same cmix); padding slots untouched.
 * col may be NULL when no row has a neighbour. */
TB_API tb_status tb_env_edge_inputs(const double *positions, const int32_t *species, int64_t n,
                                    const double *box, const int32_t *pbc, double rcut,
                                    const int64_t *slice_ptr, const int32_t *col, const int32_t *cnt,
                                    const float *cmix, const float *v, float *feat, void *stream);

/* H of the model from stored bond inputs: val (device, `precision`,
 * SELL order, padding untouched) and, when diag is not NULL, diag [n]
 * (then v [n][8], species and eps0 (device float [3]) are required). */
TB_API tb_status tb_env_forward(int64_t n, const int64_t *slice_ptr, const int32_t *cnt, const float *feat,
                                const float *v, const int32_t *species, const float *params,
                                const float *eps0, int32_t precision, void *val, void *diag,
                                void *stream);

/* Workspace bytes of tb_build_hamiltonian_env (256 + 32 n: a status word
 * and the positions as FP32 pairs). */
TB_API size_t tb_build_hamiltonian_env_workspace_size(int64_t n);

/* The same H computed straight from positions (inference at any size: no
 * stored bond inputs).  diag may be NULL; col may be NULL when no row has
 * a neighbour.  By default (tb_env_set_variant 0) the hopping network runs
 * on the 5th-generation tensor cores: every layer input (u, h1, e, h2) and
 * every weight is rounded to BF16, sums accumulate in FP32, the last layer
 * (32 -> 2) is FP32, and SiLU uses the hardware tanh approximation
 * (silu(z) = h + h tanh h, h = z/2; h1 to h3 in BF16x2 arithmetic); bond
 * vectors come from the positions split into FP32 pairs (hi + lo, exact
 * differences by TwoSum); the onsite network stays FP32.
 *   workspace  device, 256-byte aligned, at least
 *              tb_build_hamiltonian_env_workspace_size(n) bytes
 *              (TB_ERR_WORKSPACE otherwise)
 * Variant 0 synchronises `stream` (TB_ERR_TIMEOUT when a tensor-core
 * completion wait gave up); variant 1 does not. */
TB_API tb_status tb_build_hamiltonian_env(const double *positions, const int32_t *species, int64_t n,
                                          const double *box, const int32_t *pbc, double rcut,
                                          const int64_t *slice_ptr, const int32_t *col, const int32_t *cnt,
                                          const float *cmix, const float *v, const float *params,
                                          const float *eps0, int32_t precision, void *val, void *diag,
                                          void *workspace, size_t workspace_bytes, void *stream);

/* Kernel of tb_build_hamiltonian_env: 0 = tensor cores (tcgen05, BF16
 * operands; default), 1 = the FP32 pipes (the arithmetic of tb_env_forward,
 * bit for bit).  Process-wide. */
TB_API tb_status tb_env_set_variant(int32_t variant);

/* Workspace bytes of tb_env_backward. */
TB_API size_t tb_env_backward_workspace_size(int64_t n, int64_t total_elements);

/* grad (device float [TB_ENV_NPARAM]) = dL/dparams from dL/dt per real
 * element (g_val, SELL order) and dL/deps per row (g_diag [n]; rows that
 * carry no atom must have g_diag = 0 and finite v).  The forward pass is
 * recomputed; per-CTA partial sums are added in a fixed order. */
TB_API tb_status tb_env_backward(int64_t n, const int64_t *slice_ptr, const int32_t *cnt,
                                 int64_t total_elements, const float *feat, const float *v,
                                 const int32_t *species, const float *params, const float *g_val,
                                 const float *g_diag, float *grad, void *workspace,
                                 size_t workspace_bytes, void *stream);

/* Bands of a batch of periodic cells (Sec. 3: H(R) -> H(k) -> E_pre).
 * Cell c owns SELL rows [c rows_per_cell, c rows_per_cell + n_atoms)
 * (rows_per_cell a multiple of 32, n_atoms <= 64) and its neighbours must
 * lie in those rows (TB_ERR_INVALID_ARG otherwise); at most 32 neighbours
 * per row (TB_ERR_ELL_OVERFLOW).  Every stored neighbour adds
 * t e^{i k.d} with d from feat; diag (device [rows], may be NULL) adds the
 * onsite terms.  kpts: device float [n_k][3] (1/Angstrom, shared by all
 * cells).  Output: evals (device float [n_cells][n_k][n_atoms], ascending)
 * and evecs (device complex float [n_cells][n_k][n_atoms][n_atoms]:
 * component a of band b at [a][b]).  Cyclic Jacobi in FP32 until the
 * off-diagonal mass is below 1e-13 of the total (TB_ERR_NOT_CONVERGED after
 * max_sweeps sweeps).  flags: device int32 [1] scratch.  Synchronises. */
TB_API tb_status tb_bloch_bands(int32_t n_cells, int32_t n_atoms, int32_t rows_per_cell,
                                const int64_t *slice_ptr, const int32_t *col, const int32_t *cnt,
                                const float *feat, const float *val, const float *diag, int32_t n_k,
                                const float *kpts, int32_t max_sweeps, float *evals, void *evecs,
                                int32_t *flags, void *stream);

/* Eq. 3 over n_spectra spectra of n_bands bands (device float arrays
 * [n_spectra][n_bands]) with band weights w (device float [n_bands]):
 *   D = E - E_ref, S = sum w_b |D|, L = S^2 + sum w_b D^2,
 *   dLdE = 2 S w_b sign(D) + 2 w_b D  (sign(0) = 0);
 * stats (device double [3]) = {S, sum w_b D^2, L}: terms in FP32, sums in
 * FP64. */
TB_API tb_status tb_band_loss(int64_t n_spectra, int32_t n_bands, const float *evals, const float *e_ref,
                              const float *weights, float *dLdE, double *stats, void *stream);

/* Hellmann-Feynman gradients of the cells of tb_bloch_bands (same layout
 * and evecs): g_val[e] = sum_k sum_b dLdE Re(conj(psi_b[i]) psi_b[j]
 * e^{i k.d_e}) for every real element e = (i, j), g_diag[row] =
 * sum_k sum_b dLdE |psi_b[i]|^2 (0 on rows without an atom).  Valid for
 * non-degenerate bands. */
TB_API tb_status tb_band_gradient(int32_t n_cells, int32_t n_atoms, int32_t rows_per_cell,
                                  const int64_t *slice_ptr, const int32_t *col, const int32_t *cnt,
                                  const float *feat, int32_t n_k, const float *kpts, const void *evecs,
                                  const float *dLdE, float *g_val, float *g_diag, void *stream);

/* AdamW step on a flat FP32 parameter vector of n entries (same update as
 * tb_adamw_step, no BF16 copy). */
TB_API tb_status tb_adamw_flat(int64_t n, float *params, const float *grad, float *m, float *v, int64_t step,
                               double lr, double beta1, double beta2, double eps, double weight_decay,
                               void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GPUTB_H */
