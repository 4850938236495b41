// Two Chebyshev steps per launch with the matrix read once (temporal
// blocking), for the moment-doubling recursion of a single matrix.
//
// Launch `pair` computes v_m = 2 H~ v_{m-1} - v_{m-2} (stage 1) and
// v_{m+1} = 2 H~ v_m - v_{m-1} (stage 2), in place: P holds v_{m-2} and
// receives v_m, Q holds v_{m-1} and receives v_{m+1}.  The rows are cut into
// RPB-row blocks.  Stage 2 of block k may run once stage 1 has finished on
// every block it gathers v_m from (the block hull of its columns) and on
// every block that gathers v_{m-1} from block k's rows (stage 2 overwrites
// them with v_{m+1}); both sets lie in the wait interval W_k of the plan.
// Stage 2 of k then finds the
// matrix slices of block k, and v_m around it, still in L2: in one launch
// the HBM traffic is one pass over the matrix and four vector streams
// instead of two passes and six.
//
// Scheduling: a task list in global memory, in this order: stage 1 of
// block g, then the stage-2 tasks whose key is g, for g = 0 .. nb-1, where
// key_k = min(hi(W_k) + lag, nb - 1), and nb - 1 for blocks whose wait
// interval is wide (the first and last blocks of a periodic structure:
// their stage 2 runs after every stage 1).  The launch is cooperative (all
// CTAs resident) and CTA c takes list positions c, c + G, c + 2G, ... in
// order.  A stage-2 task waits only for stage-1 tasks earlier in the list
// and stage-1 tasks never wait, so the unfinished task earliest in the list
// always belongs to a resident CTA whose earlier tasks are done: it can
// proceed, and there is no deadlock.  Every wait is bounded (kPairPolls
// polls); on timeout the CTA raises flags[0] |= 4 and skips the task, which
// the host reports as TB_ERR_TIMEOUT.
//
// Coherence (the barrier idiom of CUTLASS's GenericBarrier): after stage 1
// of a block the CTA synchronises and one thread publishes the block's flag
// (value = launch epoch) with a release store; a waiter polls with relaxed
// loads, then fences (acquire) and synchronises its CTA.  Both stages read the vectors with
// ordinary (weak) loads, never the read-only path, because Q is overwritten
// during the launch (never a row that a pending stage 1 still reads).  A
// wide wait checks the per-CTA counts of finished stage-1 tasks instead of
// every flag.
//
// The per-block moment partials (four slots: <v_{m-1}|v_{m-1}>,
// <v_{m-1}|v_m>, <v_m|v_m>, <v_m|v_{m+1}>) are summed in a fixed order by
// pair_reduce_kernel, so results are bitwise reproducible although the
// block-to-CTA assignment is dynamic.
#pragma once

#include <climits>

#include "kpm_common.cuh"
#include "kpm_step.cuh"

namespace gputb {
namespace kpmdev {

constexpr long long kPairPolls = 1ll << 22;   // with 200 ns sleeps: about a second
constexpr int kBigSpan = 8192;   // wait intervals wider than this wait for every stage 1

struct PairPlan {
  const int32_t *tasks = nullptr;   // [2 nb]: >= 0 stage 1 of block t, < 0 stage 2 of block ~t
  const int2 *wait = nullptr;       // [nb] inclusive block interval W_k
  int *done = nullptr;              // [nb] epoch of the last finished stage 1
  int *cta_s1 = nullptr;            // [max_grid] stage-1 tasks finished by each CTA (cumulative)
  int64_t nb = 0;
};

__device__ __forceinline__ int ld_relaxed(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// ordinary (weak, L1-cached) load of CPT complex numbers
template <typename real, int CPT>
__device__ __forceinline__ void ld_weak(const real *p, real (&o)[2 * CPT]) {
  using V = typename Vec<real, CPT>::T;
#pragma unroll
  for (int k = 0; k < Vec<real, CPT>::kChunks; ++k) {
    V t = __ldca(reinterpret_cast<const V *>(p) + k);
    memcpy(o + k * (sizeof(V) / sizeof(real)), &t, sizeof(V));
  }
}

template <typename real, int CPT>
__device__ __forceinline__ void st_l2(real *p, const real (&v)[2 * CPT]) {
  using V = typename Vec<real, CPT>::T;
#pragma unroll
  for (int k = 0; k < Vec<real, CPT>::kChunks; ++k) {
    V t;
    memcpy(&t, v + k * (sizeof(V) / sizeof(real)), sizeof(V));
    __stcg(reinterpret_cast<V *>(p) + k, t);
  }
}

// One stage on the rows of block blk: io holds the row's v_{n-1} and receives
// v_{n+1} = alpha (H - shift) x - v_{n-1}; partials of <x|x> and <x|v_{n+1}>
// go to entry blk of slots (2 STAGE2, 2 STAGE2 + 1) of bpart.  The matrix
// is read with normal L2 priority and stage 1 stores v_m to L2 (.cg), so
// that stage 2 of the same rows finds both there; stage 2 streams.
template <typename real, typename valT, int R, int CPT, bool STAGE2>
__device__ __noinline__ void pair_stage(int64_t blk, int64_t n, const int64_t *__restrict__ slice_ptr,
                                           const int32_t *__restrict__ col, const valT *__restrict__ val,
                                           const valT *__restrict__ diag, const real *x, real *io,
                                           double *__restrict__ bpart, int64_t nb, real alpha, real shift) {
  constexpr int TPR = R / CPT;
  constexpr int RPB = kBlock / TPR;
  constexpr int kW = 16;
  const int part = threadIdx.x % TPR;
  DotAcc<real> acc[CPT], acc2[CPT];
  const int64_t i = blk * RPB + threadIdx.x / TPR;
  if (i < n) {
    const int64_t off = (i * R + part * CPT) * 2;
    real p[2 * CPT];
    ld_stream<real, CPT>(io + off, p);
    const real d = (diag ? static_cast<real>(__ldg(diag + i)) : real(0)) - shift;
    const int64_t sb = __ldg(slice_ptr + (i >> 5));
    const int w = static_cast<int>((__ldg(slice_ptr + (i >> 5) + 1) - sb) >> 5);
    const int64_t e0 = sb + (i & 31);
    real y[2 * CPT];
#pragma unroll
    for (int c = 0; c < 2 * CPT; ++c) y[c] = real(0);
    if (w <= kW) {
      int32_t j[kW];
      real h[kW];
#pragma unroll
      for (int s = 0; s < kW; ++s)
        if (s < w) {
          j[s] = __ldg(col + e0 + 32 * s);
          h[s] = static_cast<real>(__ldg(val + e0 + 32 * s));
        }
#pragma unroll
      for (int s = 0; s < kW; ++s)
        if (s < w) {
          real xv[2 * CPT];
          ld_weak<real, CPT>(x + ((int64_t)j[s] * R + part * CPT) * 2, xv);
#pragma unroll
          for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(h[s], xv[c], y[c]);
        }
    } else {
      int64_t e = e0;
      for (int s = 0; s < w; ++s, e += 32) {
        const int32_t jj = __ldg(col + e);
        const real hh = static_cast<real>(__ldg(val + e));
        real xv[2 * CPT];
        ld_weak<real, CPT>(x + ((int64_t)jj * R + part * CPT) * 2, xv);
#pragma unroll
        for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(hh, xv[c], y[c]);
      }
    }
    real xi[2 * CPT];
    ld_weak<real, CPT>(x + off, xi);
#pragma unroll
    for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(d, xi[c], y[c]);
    real o[2 * CPT];
#pragma unroll
    for (int c = 0; c < 2 * CPT; ++c) o[c] = fma(alpha, y[c], -p[c]);
    if (STAGE2)
      st_stream<real, CPT>(io + off, o);
    else
      st_l2<real, CPT>(io + off, o);
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      acc[c].add(xi[2 * c], xi[2 * c + 1], xi[2 * c], xi[2 * c + 1]);
      acc2[c].add(xi[2 * c], xi[2 * c + 1], o[2 * c], o[2 * c + 1]);
    }
  }
  double sum[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) sum[c] = acc[c].value();
  double *slot = bpart + (STAGE2 ? 2 : 0) * nb * R;
  cta_partial<R, CPT>(sum, slot + blk * R);
  __syncthreads();
#pragma unroll
  for (int c = 0; c < CPT; ++c) sum[c] = acc2[c].value();
  cta_partial<R, CPT>(sum, slot + nb * R + blk * R);
  __syncthreads();
}

// Bounded wait of a whole CTA for stage 1 on the blocks of the interval w
// (done flags equal to `epoch`; a wide interval instead waits for the
// per-CTA stage-1 counts to reach s1_target).  Polls with relaxed loads and
// a short sleep; true when the condition held, false after `polls` polls.
// Uniform across the CTA; s_tot is a shared scratch word.
__device__ __forceinline__ bool pair_wait(const PairPlan &plan, int2 w, int epoch, int64_t s1_target, long long polls,
                                          unsigned long long *s_tot) {
  const bool wide = w.y - w.x > kBigSpan;
  for (long long it = 0; it < polls; ++it) {
    bool mine = true;
    if (wide) {
      if (threadIdx.x == 0) *s_tot = 0;
      __syncthreads();
      unsigned long long tot = 0;
      for (int c = threadIdx.x; c < (int)gridDim.x; c += kBlock) tot += (unsigned)ld_relaxed(plan.cta_s1 + c);
      atomicAdd(s_tot, tot);
      __syncthreads();
      mine = *s_tot >= (unsigned long long)s1_target;
    } else {
      for (int b = w.x + (int)threadIdx.x; b <= w.y; b += kBlock) mine &= ld_relaxed(plan.done + b) == epoch;
    }
    if (__syncthreads_and(mine)) return true;
    __nanosleep(200);
  }
  return false;
}

template <typename real, typename valT, int R, int CPT>
__global__ void __launch_bounds__(kBlock, (2 * CPT * sizeof(real) >= 32) ? 2 : 4)
    cheb_pair_kernel(int64_t n, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ col,
                     const valT *__restrict__ val, const valT *__restrict__ diag, real *P, real *Q, PairPlan plan,
                     int pair, double *__restrict__ bpart, real alpha, real shift, int *flags) {
  __shared__ unsigned long long s_tot;
  const int epoch = pair + 1;
  const int64_t ntask = 2 * plan.nb;
  const int G = gridDim.x;
  // stage-1 tasks of every launch so far, for the wide waits
  const int64_t s1_target = (int64_t)epoch * plan.nb;
  int s1_mine = pair == 0 ? 0 : (threadIdx.x == 0 ? plan.cta_s1[blockIdx.x] : 0);
  for (int64_t pos = blockIdx.x; pos < ntask; pos += G) {
    const int task = __ldg(plan.tasks + pos);
    if (task >= 0) {
      const int64_t blk = task;
      pair_stage<real, valT, R, CPT, false>(blk, n, slice_ptr, col, val, diag, Q, P, bpart, plan.nb, alpha, shift);
      // pair_stage ends with __syncthreads(): every row of the block is written
      if (threadIdx.x == 0) {
        st_release(plan.done + blk, epoch);
        st_release(plan.cta_s1 + blockIdx.x, ++s1_mine);
      }
    } else {
      const int64_t blk = ~task;
      const bool ok = pair_wait(plan, plan.wait[blk], epoch, s1_target, kPairPolls, &s_tot);
      // acquire: the flags were observed with relaxed loads; the fence orders
      // this thread's later loads after them, the barrier the CTA's
      __threadfence();
      __syncthreads();
      if (ok)
        pair_stage<real, valT, R, CPT, true>(blk, n, slice_ptr, col, val, diag, P, Q, bpart, plan.nb, alpha, shift);
      else if (threadIdx.x == 0)
        atomicOr(flags, 4);
    }
  }
}

// The same two-step scheme on the bulk-copy pipeline (several threads per
// row, R >= 8): the CTA's task positions are static, so its issuing thread
// streams the next kStages tasks' matrix slices and v_{n-1} rows (stage 1:
// P rows, stage 2: Q rows -- only the task itself writes them) into the
// shared-memory ring while the CTA computes; a stage-2 task then waits for
// its stage-1 dependencies (flags) before it gathers the fresh v_m.
template <typename real, typename valT, int R, int CPT, bool STAGE2>
__device__ __forceinline__ void pair_bulk_tile(int64_t blk, int64_t n, const int64_t *__restrict__ slice_ptr,
                                               const int32_t *__restrict__ col, const valT *__restrict__ val,
                                               const valT *__restrict__ diag, const int32_t *scol, const valT *sval,
                                               const real *sprev, const real *x, real *out,
                                               double *__restrict__ bpart, int64_t nb, real alpha, real shift) {
  using G = BulkGeom<real, valT, R, CPT, 1>;
  constexpr int TPR = G::TPR, TR = G::TR;
  const int part = threadIdx.x % TPR;
  const int lr = threadIdx.x / TPR;
  DotAcc<real> acc[CPT], acc2[CPT];
  const int64_t r0 = blk * TR;
  const int64_t i = r0 + lr;
  if (i < n) {
    const int64_t k0 = r0 >> 5;
    const int64_t k1 = min((r0 + TR + 31) >> 5, (n + 31) >> 5);
    const int64_t e0 = __ldg(slice_ptr + k0);
    const bool bulk = (__ldg(slice_ptr + k1) - e0) <= G::kEl;
    real p[2 * CPT];
    memcpy(p, sprev + (lr * R + part * CPT) * 2, sizeof(p));
    const real d = (diag ? static_cast<real>(__ldg(diag + i)) : real(0)) - shift;
    const int64_t sb = __ldg(slice_ptr + (i >> 5));
    const int w = static_cast<int>((__ldg(slice_ptr + (i >> 5) + 1) - sb) >> 5);
    real y[2 * CPT];
#pragma unroll
    for (int c = 0; c < 2 * CPT; ++c) y[c] = real(0);
    if (bulk) {
      const int32_t *cs = scol + (sb - e0) + (i & 31);
      const valT *vs = sval + (sb - e0) + (i & 31);
#pragma unroll
      for (int s = 0; s < kFastW; ++s) {
        if (s < w) {
          real xv[2 * CPT];
          const real h = static_cast<real>(vs[32 * s]);
          ld_weak<real, CPT>(x + ((int64_t)cs[32 * s] * R + part * CPT) * 2, xv);
#pragma unroll
          for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(h, xv[c], y[c]);
        }
      }
    } else {
      int64_t e = sb + (i & 31);
      for (int s = 0; s < w; ++s, e += 32) {
        const int32_t jj = __ldg(col + e);
        const real hh = static_cast<real>(__ldg(val + e));
        real xv[2 * CPT];
        ld_weak<real, CPT>(x + ((int64_t)jj * R + part * CPT) * 2, xv);
#pragma unroll
        for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(hh, xv[c], y[c]);
      }
    }
    const int64_t off = (i * R + part * CPT) * 2;
    real xi[2 * CPT];
    ld_weak<real, CPT>(x + off, xi);
#pragma unroll
    for (int c = 0; c < 2 * CPT; ++c) y[c] = fma(d, xi[c], y[c]);
    real o[2 * CPT];
#pragma unroll
    for (int c = 0; c < 2 * CPT; ++c) o[c] = fma(alpha, y[c], -p[c]);
    if (STAGE2)
      st_stream<real, CPT>(out + off, o);
    else
      st_l2<real, CPT>(out + off, o);
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      acc[c].add(xi[2 * c], xi[2 * c + 1], xi[2 * c], xi[2 * c + 1]);
      acc2[c].add(xi[2 * c], xi[2 * c + 1], o[2 * c], o[2 * c + 1]);
    }
  }
  double sum[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) sum[c] = acc[c].value();
  double *slot = bpart + (STAGE2 ? 2 : 0) * nb * R;
  cta_partial<R, CPT>(sum, slot + blk * R);
  __syncthreads();
#pragma unroll
  for (int c = 0; c < CPT; ++c) sum[c] = acc2[c].value();
  cta_partial<R, CPT>(sum, slot + nb * R + blk * R);
  __syncthreads();
}

template <typename real, typename valT, int R, int CPT>
__global__ void __launch_bounds__(kBlock, bulk_min_blocks<real, R, CPT>())
    cheb_pair_bulk_kernel(int64_t n, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ col,
                          const valT *__restrict__ val, const valT *__restrict__ diag, real *P, real *Q,
                          PairPlan plan, int pair, double *__restrict__ bpart, real alpha, real shift, int *flags) {
  using G = BulkGeom<real, valT, R, CPT, 1>;
  constexpr int TR = G::TR;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ unsigned long long s_tot;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem);
  unsigned char *ring = smem + 128;
  auto s_col = [&](int st) { return reinterpret_cast<int32_t *>(ring + st * G::kStageBytes); };
  auto s_val = [&](int st) { return reinterpret_cast<valT *>(ring + st * G::kStageBytes + G::kColBytes); };
  auto s_prev = [&](int st) {
    return reinterpret_cast<real *>(ring + st * G::kStageBytes + G::kColBytes + G::kValBytes);
  };
  const int epoch = pair + 1;
  const int64_t ntask = 2 * plan.nb;
  const int grid = gridDim.x;
  const int64_t s1_target = (int64_t)epoch * plan.nb;
  int s1_mine = (pair == 0 || threadIdx.x != 0) ? 0 : plan.cta_s1[blockIdx.x];
  const int64_t my_tasks = blockIdx.x < ntask ? (ntask - 1 - blockIdx.x) / grid + 1 : 0;
  auto task_at = [&](int64_t kk) { return __ldg(plan.tasks + blockIdx.x + kk * grid); };

  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) mbar_init(full + st, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // issuing thread: matrix slices and v_{n-1} rows of local task kk
  auto issue = [&](int64_t kk) {
    const int task = task_at(kk);
    const int64_t blk = task >= 0 ? task : ~task;
    const real *prev_src = task >= 0 ? P : Q;
    const int st = static_cast<int>(kk % kStages);
    const int64_t r0 = blk * TR;
    const int64_t k0 = r0 >> 5;
    const int64_t k1 = min((r0 + TR + 31) >> 5, (n + 31) >> 5);
    const int64_t e0 = slice_ptr[k0], e1 = slice_ptr[k1];
    const bool bulk = (e1 - e0) <= G::kEl;
    const uint32_t ebytes = bulk ? static_cast<uint32_t>(e1 - e0) : 0u;
    uint32_t tx = static_cast<uint32_t>(G::kVecBytes);
    if (bulk) tx += ebytes * static_cast<uint32_t>(sizeof(int32_t) + sizeof(valT));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(full + st, tx);
    if (bulk && ebytes > 0) {
      bulk_g2s(s_col(st), col + e0, ebytes * sizeof(int32_t), full + st);
      bulk_g2s(s_val(st), val + e0, ebytes * sizeof(valT), full + st);
    }
    bulk_g2s(s_prev(st), prev_src + (size_t)r0 * R * 2, static_cast<uint32_t>(G::kVecBytes), full + st);
  };

  int64_t issued = 0;
  if (threadIdx.x == 0)
    for (; issued < my_tasks && issued < kStages; ++issued) issue(issued);
  bool ok = true;
  int64_t kk = 0;
  for (; kk < my_tasks; ++kk) {
    const int st = static_cast<int>(kk % kStages);
    const uint32_t parity = static_cast<uint32_t>((kk / kStages) & 1);
    ok = __syncthreads_and(mbar_wait_bounded(full + st, parity)) != 0;
    if (!ok) break;
    const int task = task_at(kk);
    if (task >= 0) {
      const int64_t blk = task;
      pair_bulk_tile<real, valT, R, CPT, false>(blk, n, slice_ptr, col, val, diag, s_col(st), s_val(st),
                                                s_prev(st), Q, P, bpart, plan.nb, alpha, shift);
      if (threadIdx.x == 0) {   // pair_bulk_tile ends with __syncthreads(): the block is written
        st_release(plan.done + blk, epoch);
        st_release(plan.cta_s1 + blockIdx.x, ++s1_mine);
      }
    } else {
      const int64_t blk = ~task;
      ok = pair_wait(plan, plan.wait[blk], epoch, s1_target, kPairPolls, &s_tot);
      __threadfence();   // acquire after the relaxed flag polls
      __syncthreads();
      if (!ok) break;
      pair_bulk_tile<real, valT, R, CPT, true>(blk, n, slice_ptr, col, val, diag, s_col(st), s_val(st),
                                               s_prev(st), P, Q, bpart, plan.nb, alpha, shift);
    }
    if (threadIdx.x == 0 && issued < my_tasks) issue(issued++);   // the stage of task kk is free
  }
  if (!ok) {
    // drain this CTA's own copies still in flight (bounded), then report
    if (threadIdx.x == 0) {
      atomicOr(flags, 4);
      for (int64_t q = kk; q < issued; ++q)
        mbar_wait_bounded(full + q % kStages, static_cast<uint32_t>((q / kStages) & 1));
    }
    __syncthreads();
  }
}

// ---- plan construction (once per matrix) ----------------------------------

// Hulls of block k: lo/hi = the smallest / largest block holding a column
// of block k's rows; rlo/rhi = the smallest / largest block whose rows have
// a column in block k (lo, rlo preset to INT_MAX; hi, rhi to -1).  Lanes of
// a warp with the same (column block, row block) pair share one atomic.
template <int RPB>
__global__ void pair_hull_kernel(int64_t n, const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ col,
                                 int *__restrict__ lo, int *__restrict__ hi, int *__restrict__ rlo,
                                 int *__restrict__ rhi) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i0 = i & ~int64_t(31);   // the warp's slice (launch is warp aligned)
  if (i0 >= n) return;                   // whole warp beyond the rows
  const int64_t sb = slice_ptr[i0 >> 5];
  const int w = static_cast<int>((slice_ptr[(i0 >> 5) + 1] - sb) >> 5);
  const bool real_row = i < n;
  const int own = static_cast<int>(i / RPB);
  int mn = real_row ? own : INT_MAX, mx = real_row ? own : -1;
  for (int s = 0; s < w; ++s) {
    const int b = real_row ? __ldcs(col + sb + (i & 31) + 32 * s) / RPB : -1;
    if (real_row) {
      mn = min(mn, b);
      mx = max(mx, b);
    }
    const unsigned long long key = ((unsigned long long)(unsigned)b << 32) | (unsigned)own;
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    if (real_row && (threadIdx.x & 31) == __ffs(grp) - 1) {
      atomicMin(rlo + b, own);
      atomicMax(rhi + b, own);
    }
  }
  constexpr int kSeg = RPB < 32 ? RPB : 32;   // lanes of one warp that share a row block
#pragma unroll
  for (int off = kSeg / 2; off > 0; off >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, off));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  }
  if (real_row && (threadIdx.x % kSeg) == 0) {
    atomicMin(lo + own, mn);
    atomicMax(hi + own, mx);
  }
}

// W_k = [min(lo_k, rlo_k), max(hi_k, rhi_k)], key_k, and the size of every
// task group (1 + number of keys equal to g); gsize preset to 1, gsize[nb] 0
__global__ void pair_wait_kernel(int64_t nb, int lag, const int *__restrict__ lo, const int *__restrict__ hi,
                                 const int *__restrict__ rlo, const int *__restrict__ rhi, int2 *__restrict__ wait,
                                 int *__restrict__ key, unsigned long long *__restrict__ gsize) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nb) return;
  const int wl = min(lo[k], rlo[k]), wh = max(hi[k], rhi[k]);
  wait[k] = make_int2(wl, wh);
  const int64_t last = nb - 1;
  const int64_t kk = wh - wl > kBigSpan ? last : (wh + (int64_t)lag < last ? wh + (int64_t)lag : last);
  key[k] = static_cast<int>(kk);
  atomicAdd(gsize + kk, 1ull);
}

__global__ void fill_ones_kernel(int64_t n, int64_t *__restrict__ p) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) p[k] = k + 1 < n ? 1 : 0;
}

// task list from the group offsets (exclusive scan of gsize)
__global__ void pair_tasks_kernel(int64_t nb, const int64_t *__restrict__ gstart, const int *__restrict__ key,
                                  int *__restrict__ fill, int32_t *__restrict__ tasks) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nb) return;
  tasks[gstart[k]] = static_cast<int32_t>(k);
  const int g = key[k];
  const int slot = atomicAdd(fill + g, 1);
  tasks[gstart[g] + 1 + slot] = ~static_cast<int32_t>(k);
}

// partial[s][u][r] (s = 0..3, u < units) = sum of the block partials of
// chunk u of the blocks, in block order
__global__ void pair_reduce_kernel(const double *__restrict__ bpart, int64_t nb, int R, int units,
                                   double *__restrict__ partial, int64_t slot_stride) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4ll * units * R) return;
  const int r = static_cast<int>(t % R);
  const int u = static_cast<int>((t / R) % units);
  const int s = static_cast<int>(t / ((int64_t)R * units));
  const int64_t b0 = nb * u / units, b1 = nb * (u + 1) / units;
  const double *p = bpart + (int64_t)s * nb * R + r;
  double acc = 0.0;
  for (int64_t b = b0; b < b1; ++b) acc += p[b * R];
  partial[s * slot_stride + (int64_t)u * R + r] = acc;
}

}  // namespace kpmdev
}  // namespace gputb
